"""Batched form: many graphs in one launch per round equal the same graphs alone (GPU).

Each round gives every graph a mixed batch (insertion half, then deletion half).
After every round each graph's levels, counters and work counts must equal those
of a separate handle that applied the same halves with plds_batch_insert and
plds_batch_delete, and a sample of graphs is checked against the CPU oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_03824_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("valid", "self_loops", "duplicates", "filtered", "rounds", "moves", "visits", "dl_evals", "dl_visits")


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds
    return plds


def _graphs(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(200), np.log(6000))))
        deg = rng.uniform(4, 32)
        gamma = rng.uniform(2.1, 2.8)
        out.append((n, W.chung_lu(n, int(n * deg / 2), gamma, seed=seed * 1000 + i)))
    return out


def _round(rng, e, present, n, r):
    """A mixed batch of 1-10% of the graph's edges, with noise."""
    k = max(1, int(rng.uniform(0.01, 0.10) * e.shape[0]))
    ins = e[rng.choice(e.shape[0], size=min(k, e.shape[0]), replace=False)]
    pres = np.array(sorted(present), np.int64).reshape(-1, 2) if present else np.zeros((0, 2), np.int64)
    kd = min(k // 2, pres.shape[0])
    dele = pres[rng.choice(pres.shape[0], size=kd, replace=False)] if kd else pres[:0]
    ins = W.noisy_batch(ins, n, seed=r, self_loops=2, dups=3, reversed_frac=0.3)
    dele = W.noisy_batch(dele.astype(np.int32), n, seed=r + 7, dups=2, reversed_frac=0.3)
    return ins, dele


def test_set_rounds_equal_single_graphs(P):
    graphs = _graphs(48, seed=3)
    S = P.PLDSSet([n for n, _ in graphs])
    alone = [P.PLDS(n) for n, _ in graphs]
    orc = {i: O.OraclePLDS(graphs[i][0]) for i in (0, 5, 17, 47)}
    present = [set() for _ in graphs]
    rng = np.random.default_rng(11)
    for r in range(6):
        halves = [_round(rng, e, present[i], n, 100 * r + i) for i, (n, e) in enumerate(graphs)]
        edges, offs = S.pack(halves)
        S.update(edges if r % 2 else torch.from_numpy(edges).cuda(), offs)
        for i, (ins, dele) in enumerate(halves):
            alone[i].insert(ins)
            s1 = alone[i].stats()
            alone[i].delete(dele)
            s2 = alone[i].stats()
            gs = S.graphs[i].stats()
            assert np.array_equal(S.graphs[i].levels(), alone[i].levels()), (r, i)
            for a, b in zip(S.graphs[i].counters(), alone[i].counters()):
                assert np.array_equal(a, b), (r, i)
            for k in KEYS:
                assert gs[k] == s1[k] + s2[k], (r, i, k)
            for u, v in ins:
                if u != v:
                    present[i].add((min(u, v), max(u, v)))
            for u, v in dele:
                present[i].discard((min(u, v), max(u, v)))
            if i in orc:
                orc[i].insert(ins)
                orc[i].delete(dele)
                assert np.array_equal(S.graphs[i].levels(), orc[i].levels()), (r, i)
    S.close()
    for g in alone:
        g.close()


def test_set_rejects_bad_ids(P):
    S = P.PLDSSet([100, 200])
    halves = [(np.array([[0, 1], [2, 3]], np.int32), np.zeros((0, 2), np.int32)),
              (np.array([[0, 250]], np.int32), np.zeros((0, 2), np.int32))]
    edges, offs = S.pack(halves)
    assert S.update(edges, offs, check=False) == P.PLDS_EINVAL
    S.close()


def test_set_knobs_never_change_results_and_autotune(P):
    """Thread cutoff, block cutoff and load factor change only speed: a set under
    extreme knobs (and under the knobs the autotuner picks on a sample of the same
    workload) ends every round with the same levels as the default set."""
    graphs = _graphs(24, seed=8)
    ns = [n for n, _ in graphs]
    rng = np.random.default_rng(4)
    present = [set() for _ in graphs]
    rounds = []
    for r in range(5):
        halves = [_round(rng, e, present[i], n, 100 * r + i) for i, (n, e) in enumerate(graphs)]
        for i, (ins, dele) in enumerate(halves):
            for u, v in ins:
                if u != v:
                    present[i].add((min(u, v), max(u, v)))
            for u, v in dele:
                present[i].discard((min(u, v), max(u, v)))
        rounds.append(P.PLDSSet.pack(halves))
    dev = [(torch.from_numpy(e).cuda(), o) for e, o in rounds]
    ref = P.PLDSSet(ns)
    want = []
    for e, o in dev:
        ref.update(e, o)
        want.append([g.levels().copy() for g in ref.graphs])
    ref.close()
    tuned = P.PLDSSet(ns)
    best = tuned.autotune(dev[:3], timed_from=1, max_trials=8)
    assert best["thread_max_cap"] in (4, 8, 16, 32, 64)
    assert best["block_cap"] in (1024, 2048, 4096, 8192, 16384)
    assert (best["load_num"], best["load_den"]) in ((1, 2), (5, 8), (3, 4), (7, 8))
    assert best["list_cap"] in (128, 256, 1024, 1 << 30)
    extreme = P.PLDSSet(ns)
    extreme.tune(thread_max_cap=4, block_cap=4, load_num=1, load_den=2, list_cap=32)
    for r, (e, o) in enumerate(dev):
        for S in (tuned, extreme):
            S.update(e, o)
            for i, g in enumerate(S.graphs):
                assert np.array_equal(g.levels(), want[r][i]), (r, i, best)
    tuned.close()
    extreme.close()
