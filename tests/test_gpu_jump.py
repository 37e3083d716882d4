"""Jump variant of the insertion rounds on the GPU vs the oracle's jump mode.

The Experiments section's implementation computes, for the vertices it moves up,
a desire-level by a filter and sort instead of moving them one level per round.
Both sides read it the same way (each round, every violator of Invariant 1 on the
lowest level holding one moves straight to the lowest level above it where it
satisfies Invariant 1 with every other vertex where it is), so after every batch
the levels, the counters and the variant's own rounds / moves / visits must equal
the oracle's (integers: exact), and the levels must equal Algorithm 2's.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03824_gb300 import workloads as W
from test_gpu_parity import assert_same

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

JUMP_STATS = ("valid", "rounds", "moves", "visits", "dl_evals", "dl_visits")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds
    return plds


def check(g, o, what):
    assert_same(g, o, what)
    gs, os_ = g.stats(), o.stats()
    for k in JUMP_STATS:
        assert gs[k] == os_[k], f"{what}: stat {k} gpu={gs[k]} oracle={os_[k]}"


def run_stream(P, n, e, batch, delta=0.4, lam=3.0, lpg=0, dels=True, device=False):
    g = P.PLDS(n, delta, lam, lpg, jump=True)
    o = O.OraclePLDS(n, delta, lam, lpg, flags=O.JUMP)
    a = O.OraclePLDS(n, delta, lam, lpg)  # Algorithm 2: the same levels
    rounds_jump = rounds_alg2 = 0
    for i, b in enumerate(W.batches(W.shuffled(e, 11), batch)):
        g.insert(torch.from_numpy(b).cuda() if device else b)
        assert o.insert(b) == 0 and a.insert(b) == 0
        check(g, o, f"ins {i}")
        assert np.array_equal(g.levels(), a.levels()), f"ins {i}: levels differ from Algorithm 2's"
        rounds_jump += o.stats()["rounds"]
        rounds_alg2 += a.stats()["rounds"]
    if dels:
        for i, b in enumerate(W.batches(W.shuffled(e, 12), batch)):
            g.delete(b)
            assert o.delete(b) == 0
            check(g, o, f"del {i}")
    g.close()
    return rounds_jump, rounds_alg2


def test_jump_small_config_every_batch(P):
    """Chung-Lu n=10^4, m=5*10^4, gamma=2.5, batches of 1000 (Ins, then Del)."""
    rj, ra = run_stream(P, 10_000, W.chung_lu(10_000, 50_000, 2.5, seed=1), 1000)
    assert rj <= ra


def test_jump_rmat16_every_batch(P):
    """R-MAT scale 16 (0.9 M edges) in batches of 58k: hubs take the block-wide target
    and apply paths; device-resident inputs."""
    e = W.rmat(16, 16, seed=1)
    rj, ra = run_stream(P, 1 << 16, e, 58_000, dels=True, device=True)
    assert rj < ra


@pytest.mark.parametrize("delta,lam", [(0.2, 3.0), (1.6, 12.0), (6.4, 96.0)])
def test_jump_parameter_grid(P, delta, lam):
    n = 4000
    run_stream(P, n, W.chung_lu(n, 30_000, 2.2, seed=5), 3000, delta=delta, lam=lam)


def test_jump_toy_groups_and_star(P):
    """Three levels per group (the worked examples' size) and a 3000-leaf star plus
    a 60-clique: long climbs and a large table in one round."""
    n = 4000
    rng = np.random.default_rng(4)
    star = np.stack([np.zeros(3000, np.int32), np.arange(1, 3001, dtype=np.int32)], 1)
    cl = np.array([(3100 + i, 3100 + j) for i in range(60) for j in range(i + 1, 60)], np.int32)
    e = np.concatenate([star, cl, W.erdos_renyi(n, 6000, seed=9)])
    e = np.unique(np.sort(e, 1), axis=0)
    e = e[e[:, 0] != e[:, 1]]
    e = e[rng.permutation(e.shape[0])].astype(np.int32)
    run_stream(P, n, e, 2500, lpg=3)
