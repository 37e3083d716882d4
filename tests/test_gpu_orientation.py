"""Low out-degree orientation (Section "O(alpha) Out-Degree Orientation",
Algorithm 5) on the GPU against the CPU oracle.

After every batch: the tail of every queried edge (present, absent, invalid), every
vertex's out-degree, the flipped edges F and the oriented updates J of the batch
must equal the oracle's (F and J compared as sets: the GPU returns them unordered).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03824_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds
    return plds


def _sorted_pairs(a):
    a = np.asarray(a, np.int64).reshape(-1, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def _compare(g, o, rng, n, what):
    cur = o.edges()
    q = [cur[rng.integers(0, cur.shape[0], size=min(500, cur.shape[0]))]] if cur.shape[0] else []
    q.append(rng.integers(0, n, size=(200, 2)).astype(np.int32))          # mostly absent
    q.append(np.array([[0, 0], [-1, 3], [2, n]], np.int32))              # invalid
    qe = np.ascontiguousarray(np.concatenate(q).astype(np.int32))
    assert np.array_equal(g.orient(qe), o.orient(qe)), f"{what}: tails differ"
    assert np.array_equal(g.out_degrees(), o.out_degrees()), f"{what}: out-degrees differ"
    assert np.array_equal(_sorted_pairs(g.flips()), _sorted_pairs(o.flips())), f"{what}: F differs"
    assert np.array_equal(_sorted_pairs(g.oriented_updates()), _sorted_pairs(o.oriented_updates())), \
        f"{what}: J differs"


def test_orientation_matches_oracle_every_batch(P):
    n = 3000
    rng = np.random.default_rng(8)
    e = W.chung_lu(n, 30_000, 2.2, seed=8)
    g, o = P.PLDS(n), O.OraclePLDS(n)
    g.set_tuning(track_orientation=1)
    o.track(True)
    for step in range(12):
        pick = e[rng.choice(e.shape[0], size=int(rng.integers(100, 5000)), replace=False)]
        ins = W.noisy_batch(pick, n, seed=step, self_loops=3, dups=20, reversed_frac=0.4)
        g.insert(ins)
        o.insert(ins)
        _compare(g, o, rng, n, f"step {step} ins")
        cur = o.edges()
        k = int(rng.integers(0, max(1, cur.shape[0] // 2)))
        dl = cur[rng.choice(cur.shape[0], size=k, replace=False)] if k else cur[:0]
        g.delete(dl)
        o.delete(dl)
        _compare(g, o, rng, n, f"step {step} del")
    g.close()


def test_orientation_rmat_and_tracking_off(P):
    scale = 14
    n = 1 << scale
    e = W.rmat(scale, 16, seed=3)
    rng = np.random.default_rng(1)
    g, o = P.PLDS(n), O.OraclePLDS(n)
    with pytest.raises(P.PldsError):
        g.flips()  # nothing tracked yet
    g.set_tuning(track_orientation=1)
    o.track(True)
    for i, b in enumerate(W.batches(W.shuffled(e, 5), 40_000)):
        g.insert(b)
        o.insert(b)
        _compare(g, o, rng, n, f"ins {i}")
    for i, b in enumerate(list(W.batches(W.shuffled(e, 6), 40_000))[:3]):
        g.delete(b)
        o.delete(b)
        _compare(g, o, rng, n, f"del {i}")
    g.set_tuning(track_orientation=0)
    g.insert(e[:10])
    with pytest.raises(P.PldsError):
        g.flips()
    g.close()
