"""CUDA path vs the CPU oracle (GPU tests; every call goes through the C ABI).

Levels, deg/up/up* counters, coreness exponents and the per-batch work counts
(rounds, moves, neighbour visits, desire-level evaluations) must be identical to
the oracle's after every batch: all of them are integers decided by exact integer
arithmetic on both sides.  The coreness estimate itself is a double
(1+delta)^g; both sides form it from the same integer exponent, so it is compared
with a relative tolerance of 1e-12 (a few ulps of at most ~60 multiplications).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03824_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STAT_KEYS = ("valid", "self_loops", "duplicates", "filtered", "rounds", "moves", "visits", "dl_evals",
             "dl_visits")
REL_TOL = 1e-12


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds
    return plds


def assert_same(g, o, what=""):
    lv, olv = g.levels(), o.levels()
    if not np.array_equal(lv, olv):
        bad = np.nonzero(lv != olv)[0]
        raise AssertionError(f"{what}: {bad.size} levels differ, first {bad[:5]} gpu={lv[bad[:5]]} "
                             f"oracle={olv[bad[:5]]}")
    d, u, s = g.counters()
    od, ou, os_ = o.counters()
    assert np.array_equal(d, od), f"{what}: deg differs"
    assert np.array_equal(u, ou), f"{what}: up differs"
    assert np.array_equal(s, os_), f"{what}: up* differs"
    assert np.array_equal(g.coreness_exponent(), o.coreness_exponent()), f"{what}: exponent differs"
    ge, oe = g.coreness(), o.coreness()
    assert np.allclose(ge, oe, rtol=REL_TOL, atol=0), f"{what}: coreness differs"


def assert_stats(g, o, what=""):
    gs, os_ = g.stats(), o.stats()
    for k in STAT_KEYS:
        assert gs[k] == os_[k], f"{what}: stat {k} gpu={gs[k]} oracle={os_[k]}"


def test_tables_match_oracle(P):
    for n, d, lam, lpg in [(10_000, 0.4, 3.0, 0), (1 << 20, 0.4, 3.0, 0), (41_700_000, 0.4, 3.0, 0),
                           (1000, 1.0, 3.0, 3), (5000, 0.2, 12.0, 0), (77, 3.2, 96.0, 0), (1, 0.4, 3.0, 0)]:
        g = P.PLDS(n, d, lam, lpg)
        T = O.tables(n, d, lam, lpg)
        assert (g.t, g.Lg, g.G, g.K) == (T["t"], T["Lg"], T["G"], T["K"])
        up, dn = g.tables()
        assert np.array_equal(up, T["upmax"]) and np.array_equal(dn, T["dnmin"])
        g.close()


def test_small_config_every_batch(P):
    """Chung-Lu n=10^4, m=5*10^4, gamma=2.5: 50 Ins batches of 1000, then 50 Del batches."""
    n = 10_000
    e = W.chung_lu(n, 50_000, 2.5, seed=1)
    g, o = P.PLDS(n), O.OraclePLDS(n)
    for i, b in enumerate(W.batches(W.shuffled(e, 11), 1000)):
        g.insert(b)
        assert o.insert(b) == 0
        assert_same(g, o, f"ins {i}")
        assert_stats(g, o, f"ins {i}")
    dels = W.shuffled(o.edges(), 12)
    for i, b in enumerate(list(W.batches(dels, 1000))[:50]):
        g.delete(torch.from_numpy(b).cuda())
        assert o.delete(b) == 0
        assert_same(g, o, f"del {i}")
        assert_stats(g, o, f"del {i}")
    g.close()


@pytest.mark.parametrize("seed", [1, 2])
def test_mixed_noisy_batches(P, seed):
    """Update(B) = insert half then delete half; batches carry self-loops, duplicates,
    reversed pairs, inserts of present and deletes of absent edges."""
    n = 3000
    rng = np.random.default_rng(seed)
    e = W.chung_lu(n, 30_000, 2.2, seed=seed)
    g, o = P.PLDS(n), O.OraclePLDS(n)
    present = np.zeros((0, 2), np.int32)
    for step in range(16):
        pick = e[rng.choice(e.shape[0], size=int(rng.integers(100, 4000)), replace=False)]
        ins = W.noisy_batch(pick, n, seed=step, self_loops=5, dups=50, reversed_frac=0.5)
        g.insert(ins)
        assert o.insert(ins) == 0
        assert_same(g, o, f"step {step} ins")
        assert_stats(g, o, f"step {step} ins")
        cur = o.edges()
        k = int(rng.integers(0, max(1, cur.shape[0] // 2)))
        dl = cur[rng.choice(cur.shape[0], size=k, replace=False)] if k else cur[:0]
        dl = W.noisy_batch(np.concatenate([dl, pick[:50]]), n, seed=100 + step, self_loops=3, dups=20,
                           reversed_frac=0.5)
        g.delete(dl)
        assert o.delete(dl) == 0
        assert_same(g, o, f"step {step} del")
        assert_stats(g, o, f"step {step} del")
    g.close()


def test_invalid_ids_rejected_without_change(P):
    n = 500
    e = W.erdos_renyi(n, 3000, seed=3)
    g, o = P.PLDS(n), O.OraclePLDS(n)
    g.insert(e)
    o.insert(e)
    before = g.levels().copy()
    bad = np.concatenate([e[:10], np.array([[0, n]], np.int32)])
    assert g.insert(bad, check=False) == P.PLDS_EINVAL
    assert g.delete(np.array([[-1, 2]], np.int32), check=False) == P.PLDS_EINVAL
    assert np.array_equal(g.levels(), before)
    assert_same(g, o, "after rejected batches")
    g.delete(e[:1000])
    o.delete(e[:1000])
    assert_same(g, o, "usable after rejection")
    g.close()


def test_degenerate_inputs(P):
    g = P.PLDS(1)
    g.insert(np.zeros((0, 2), np.int32))
    g.insert(np.array([[0, 0], [0, 0]], np.int32))
    assert g.levels()[0] == 0 and g.coreness()[0] == 0.0
    assert g.stats()["self_loops"] == 2
    g.close()
    n = 64
    g, o = P.PLDS(n), O.OraclePLDS(n)
    loops = np.stack([np.arange(n), np.arange(n)], 1).astype(np.int32)
    g.insert(loops)
    o.insert(loops)
    assert_same(g, o, "self-loops only")
    g.delete(np.array([[1, 2]], np.int32))  # absent edge
    assert g.stats()["filtered"] == 1
    g.close()


def test_star_hub_and_clique(P):
    """A hub with 30k leaves (multi-chunk tables, several regrowths) and a 80-clique
    (a long climb through many groups' levels), inserted and then deleted."""
    n = 40_000
    star = np.stack([np.zeros(30_000, np.int32), np.arange(1, 30_001, dtype=np.int32)], 1)
    cl = np.array([(a, b) for a in range(30_001, 30_081) for b in range(a + 1, 30_081)], np.int32)
    cross = np.stack([np.zeros(80, np.int32), np.arange(30_001, 30_081, dtype=np.int32)], 1)
    g, o = P.PLDS(n), O.OraclePLDS(n)
    for b in (star[:1000], star[1000:], cl, cross):
        g.insert(b)
        o.insert(b)
        assert_same(g, o, "insert")
        assert_stats(g, o, "insert")
    for b in (cl[::2], star[::3], cross, cl[1::2], star):
        g.delete(b)
        o.delete(b)
        assert_same(g, o, "delete")
        assert_stats(g, o, "delete")
    g.close()


@pytest.mark.parametrize("scale,batch", [(14, 20_000), (16, 100_000)])
def test_rmat_every_batch(P, scale, batch):
    """R-MAT (a,b,c,d)=(.57,.19,.19,.05), edge factor 16: Ins then Del in batches."""
    n = 1 << scale
    e = W.rmat(scale, 16, seed=scale)
    g, o = P.PLDS(n), O.OraclePLDS(n)
    for i, b in enumerate(W.batches(W.shuffled(e, 1), batch)):
        g.insert(b)
        o.insert(b)
        assert_same(g, o, f"ins {i}")
        assert_stats(g, o, f"ins {i}")
    for i, b in enumerate(W.batches(W.shuffled(e, 2), batch)):
        g.delete(b)
        o.delete(b)
        assert_same(g, o, f"del {i}")
        assert_stats(g, o, f"del {i}")
    assert g.levels().max() == 0
    g.close()


@pytest.mark.parametrize("delta,lam,heuristic", [(0.2, 12.0, False), (0.8, 6.0, False), (1.6, 48.0, False),
                                                  (3.2, 96.0, False), (6.4, 24.0, False), (0.4, 3.0, True),
                                                  (1.6, 3.0, True)])
def test_parameter_grid_every_batch(P, delta, lam, heuristic):
    """Other points of the experiments' delta / lambda grid, and the heuristic
    coefficient 1.1: Chung-Lu n = 5000, Ins then Del batches, equal to the oracle
    after every batch (tables included)."""
    _grid_case(P, delta, lam, heuristic)


def test_many_groups_every_batch(P):
    """delta = 0.03 at n = 5000: 290 groups of 1156 levels, so the desire-level's
    group and window histograms no longer share one warp's scratch and every
    evaluation takes its two-scan path; equal to the oracle after every batch."""
    assert O.tables(5000, 0.03, 3.0)["G"] == 290
    _grid_case(P, 0.03, 3.0, False)


def _grid_case(P, delta, lam, heuristic):
    n = 5000
    e = W.chung_lu(n, 30_000, 2.3, seed=31)
    flags = O.HEURISTIC if heuristic else 0
    g = P.PLDS(n, delta, lam, heuristic=heuristic)
    o = O.OraclePLDS(n, delta, lam, flags=flags)
    T = O.tables(n, delta, lam, flags=flags)
    up, dn = g.tables()
    assert np.array_equal(up, T["upmax"]) and np.array_equal(dn, T["dnmin"])
    for i, b in enumerate(W.batches(W.shuffled(e, 3), 4000)):
        g.insert(b)
        o.insert(b)
        assert_same(g, o, f"ins {i}")
        assert_stats(g, o, f"ins {i}")
    for i, b in enumerate(W.batches(W.shuffled(e, 4), 4000)):
        g.delete(b)
        o.delete(b)
        assert_same(g, o, f"del {i}")
        assert_stats(g, o, f"del {i}")
    g.close()


def test_pldsopt_every_batch(P):
    """PLDSOpt (ceil(log_{1+delta} m / 50) levels per group, here 1): the same batch
    rules on fewer levels; levels, counters and work counts equal the oracle's with
    the same group size after every batch, and the oracle's invariant checks pass."""
    scale, batch = 16, 100_000
    n = 1 << scale
    e = W.rmat(scale, 16, seed=scale)
    lg = P.opt_levels_per_group(e.shape[0])
    assert lg == O.opt_levels_per_group(e.shape[0]) == 1
    g, o = P.PLDS(n, levels_per_group=lg), O.OraclePLDS(n, levels_per_group=lg)
    assert g.Lg == lg and g.K == g.G * lg
    for i, b in enumerate(W.batches(W.shuffled(e, 1), batch)):
        g.insert(b)
        o.insert(b)
        assert o.check() == 0
        assert_same(g, o, f"opt ins {i}")
        assert_stats(g, o, f"opt ins {i}")
    for i, b in enumerate(W.batches(W.shuffled(e, 2), batch)):
        g.delete(b)
        o.delete(b)
        assert o.check() == 0
        assert_same(g, o, f"opt del {i}")
        assert_stats(g, o, f"opt del {i}")
    g.close()


def test_tuning_never_changes_results(P):
    n = 1 << 13
    e = W.rmat(13, 16, seed=5)
    ref = None
    for tune in (dict(), dict(thread_max_cap=4, load_num=1, load_den=2, block_threads=256, block_cap=4, list_cap=8),
                 dict(thread_max_cap=64, load_num=7, load_den=8, block_threads=512, blocks_per_sm=2,
                      block_cap=16384, list_cap=1 << 30)):
        g = P.PLDS(n)
        if tune:
            g.set_tuning(**tune)
        out = []
        for b in W.batches(W.shuffled(e, 3), 7000):
            g.insert(b)
            out.append(g.levels().copy())
        for b in W.batches(W.shuffled(e, 4)[: e.shape[0] // 2], 7000):
            g.delete(b)
            out.append(g.levels().copy())
        g.close()
        if ref is None:
            ref = out
        else:
            assert all(np.array_equal(a, b) for a, b in zip(ref, out))


def test_host_and_device_buffers(P):
    n = 5000
    e = W.chung_lu(n, 20_000, 2.4, seed=9)
    g = P.PLDS(n, torch_allocator=False)  # library's own cudaMallocAsync path
    g.insert(torch.from_numpy(e).cuda())
    h_lv = g.levels()
    d_lv = torch.empty(n, dtype=torch.int32, device="cuda")
    g.levels(d_lv)
    torch.cuda.synchronize()
    assert np.array_equal(h_lv, d_lv.cpu().numpy())
    d_c = torch.empty(n, dtype=torch.float64, device="cuda")
    g.coreness(d_c)
    torch.cuda.synchronize()
    assert np.array_equal(g.coreness(), d_c.cpu().numpy())
    g.close()


def test_bounded_wait_reports_timeout(P):
    """Block 0 sleeps 50 ms before its first barrier while the wait limit is 1 ms:
    the barrier gives up, the call returns PLDS_ETIMEOUT, the handle is poisoned, and
    the device stays usable for a fresh handle."""
    n = 1000
    e = W.erdos_renyi(n, 4000, seed=1)
    g = P.PLDS(n)
    g.set_tuning(test_delay_us=50_000)
    g.set_wait_limit(1_000_000)
    assert g.insert(e, check=False) == P.PLDS_ETIMEOUT
    assert g.insert(e, check=False) == P.PLDS_EPOISONED
    g.close()
    g2, o = P.PLDS(n), O.OraclePLDS(n)
    g2.insert(e)
    o.insert(e)
    assert_same(g2, o, "fresh handle after timeout")
    g2.close()


def test_rejected_insertion_leaves_no_trace(P):
    """A rejected insertion batch whose other edges are new and valid: the next
    batches grow the tables exactly as on a graph that never saw it (same pool use,
    same levels and counters as the oracle)."""
    n = 3000
    e = W.erdos_renyi(n, 20_000, seed=41)
    a, b, o = P.PLDS(n), P.PLDS(n), O.OraclePLDS(n)
    for h in (a, b):
        h.insert(e[:8000])
    o.insert(e[:8000])
    bad = np.concatenate([e[8000:14000], np.array([[5, n + 3]], np.int32)])
    assert a.insert(bad, check=False) == P.PLDS_EINVAL
    for h in (a, b):
        h.insert(e[8000:])
    o.insert(e[8000:])
    assert_same(a, o, "after the rejected batch")
    assert a.stats()["pool_slots_used"] == b.stats()["pool_slots_used"]
    a.close()
    b.close()


def test_single_handle_autotune(P):
    """plds_autotune on a sample stream: the handle's graph is untouched, the knobs
    picked are candidates of the search, and results with them still equal the
    oracle's."""
    n = 20_000
    e = W.shuffled(W.chung_lu(n, 100_000, 2.3, seed=12), 3)
    g, o = P.PLDS(n), O.OraclePLDS(n)
    g.insert(e[:40_000])
    o.insert(e[:40_000])
    before = g.levels().copy()
    sample = [("ins", e[:30_000]), ("ins", torch.from_numpy(e[30_000:60_000]).cuda()), ("del", e[:10_000])]
    knobs = g.autotune(sample, timed_from=1, max_trials=6)
    assert np.array_equal(g.levels(), before)
    assert knobs["thread_max_cap"] in (4, 8, 16, 32, 64)
    assert knobs["block_cap"] in (1024, 2048, 4096, 8192, 16384)
    assert (knobs["load_num"], knobs["load_den"]) in ((1, 2), (5, 8), (3, 4), (7, 8))
    g.insert(e[40_000:])
    o.insert(e[40_000:])
    assert_same(g, o, "after autotune")
    g.delete(e[::2])
    o.delete(e[::2])
    assert_same(g, o, "after autotune, deletions")
    g.close()
