"""Serving form (GPU).

Unchanged boundaries (merging off): a mixed stream of insertion and deletion
batches of uneven sizes (10 .. 20,000 edges, from device, pinned and pageable host
buffers) with coreness queries in between is submitted faster than it is served,
so requests wait for ring slots and run back to back.  Every request's work
counts, every query's values, and the final levels must equal those of a second
graph that applies the same requests with plds_batch_insert / plds_batch_delete /
plds_coreness; a dense batch forces the adjacency pool to grow while the loop runs.

Continuous batching (merging on): requests that queue behind a long one are
applied together.  The logged schedule (batch_first, batch_size of every result)
replayed batch by batch through the CPU oracle must give bit-identical levels,
counts and query values; a request with a bad id is rejected alone; and every
query's estimates, in the mix and with the same requests applied alone, are within
the paper's bound (2 + 3/lambda)(1 + delta) of the exact coreness both ways.
"""
from fractions import Fraction

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


def test_served_stream_equals_separate_calls(P):
    n = 30_000
    e = W.chung_lu(n, 200_000, 2.3, seed=17)
    rng = np.random.default_rng(5)
    reqs = []  # (op, edges)
    present = np.zeros((0, 2), np.int32)
    pos = 0
    order = W.shuffled(e, 3)
    for k in range(60):
        if k % 7 == 6:
            reqs.append((2, None))
            continue
        size = int(np.exp(rng.uniform(np.log(10), np.log(20_000))))
        if rng.random() < 0.6 or present.shape[0] < size:
            b = order[pos:pos + size]
            pos += size
            reqs.append((0, W.noisy_batch(b, n, seed=k, self_loops=1, dups=2, reversed_frac=0.2)))
            present = np.concatenate([present, b])
        else:
            idx = rng.choice(present.shape[0], size=size, replace=False)
            reqs.append((1, present[idx]))
            present = np.delete(present, idx, axis=0)
    # a dense block (1000 vertices, ~250k edges) whose tables overflow the initial pool
    # while the loop runs
    blk = W.erdos_renyi(1000, 300_000, seed=9)
    reqs.insert(30, (0, blk))
    served, plain = P.PLDS(n), P.PLDS(n)
    sv = P.Server(served, slots=4, max_batch=400_000, merge_max_edges=0)
    outs, expect, kinds = {}, {}, {}
    for k, (op, b) in enumerate(reqs):
        if op == 2:
            out = torch.empty(n, dtype=torch.float64, device="cuda") if k % 2 else np.zeros(n)
            t = sv.submit(2, out=out)
            outs[t] = out
            expect[t] = plain.coreness()
        else:
            src = b
            if k % 3 == 1:
                src = torch.from_numpy(b).cuda()
            elif k % 3 == 2:
                src = torch.from_numpy(b).pin_memory()
            t = sv.submit(op, edges=src)
            (plain.insert if op == 0 else plain.delete)(b)
            expect[t] = plain.stats()
        kinds[t] = op
    sv.drain()
    results = {r["ticket"]: r for r in sv.poll(4096)}
    assert sorted(results) == list(range(len(reqs)))
    for t, r in results.items():
        assert r["status"] == 0, (t, r)
        if kinds[t] == 2:
            got = outs[t].cpu().numpy() if hasattr(outs[t], "cpu") else outs[t]
            assert np.array_equal(got, expect[t]), t
        else:
            for key in ("valid", "rounds", "moves"):
                assert r[key] == expect[t][key], (t, key, r[key], expect[t][key])
    sv.close()
    assert np.array_equal(served.levels(), plain.levels())
    for a, b in zip(served.counters(), plain.counters()):
        assert np.array_equal(a, b)
    assert served.stats()["pool_grows"] >= 1
    served.close()
    plain.close()


def _stream(n, seed, count, bad_at=()):
    """Mixed requests on a Chung-Lu graph: (op, edges) with op 2 = coreness query."""
    e = W.chung_lu(n, 200_000, 2.3, seed=seed)
    rng = np.random.default_rng(seed)
    order = W.shuffled(e, seed + 1)
    reqs, present, pos = [], np.zeros((0, 2), np.int32), 0
    for k in range(count):
        if k % 9 == 8:
            reqs.append((2, None))
            continue
        size = int(np.exp(rng.uniform(np.log(10), np.log(5_000))))
        if k in bad_at:
            b = order[pos:pos + size].copy()
            b[size // 2, 1] = n  # out of range: the request is rejected alone
            reqs.append((0, b))
        elif rng.random() < 0.6 or present.shape[0] < size:
            b = order[pos:pos + size]
            pos += size
            reqs.append((0, W.noisy_batch(b, n, seed=k, self_loops=1, dups=2, reversed_frac=0.3)))
            present = np.concatenate([present, b])
        else:
            idx = rng.choice(present.shape[0], size=size, replace=False)
            reqs.append((1, present[idx]))
            present = np.delete(present, idx, axis=0)
    return reqs


def _within_bound(est, core, delta=0.4, lam=3.0):
    c = float((2 + Fraction(3) / Fraction(round(lam * 10**6), 10**6)) * (1 + Fraction(round(delta * 10**6), 10**6)))
    zero = core == 0
    if not np.array_equal(est == 0, zero):
        return False
    k, kh = core[~zero].astype(np.float64), est[~zero]
    return bool(np.all(k <= c * kh * (1 + 1e-12)) and np.all(kh <= c * k * (1 + 1e-12)))


def test_merged_schedule_replays_on_oracle(P):
    n = 30_000
    reqs = _stream(n, 23, 90, bad_at=(13, 40))
    # a long first request so that the rest queue up behind it and get merged
    reqs.insert(0, (0, W.erdos_renyi(1000, 300_000, seed=4)))
    served = P.PLDS(n)
    sv = P.Server(served, slots=32, max_batch=400_000)
    outs, kinds, src = {}, {}, {}
    for k, (op, b) in enumerate(reqs):
        if op == 2:
            out = np.zeros(n)
            t = sv.submit(2, out=out)
            outs[t] = out
        else:
            buf = torch.from_numpy(b).pin_memory() if k % 2 else torch.from_numpy(b).cuda()
            t = sv.submit(op, edges=buf)
            src[t] = b
        kinds[t] = op
    sv.drain()
    res = {r["ticket"]: r for r in sv.poll(4096)}
    sv.close()
    assert sorted(res) == list(range(len(reqs)))
    assert max(r["batch_size"] for r in res.values()) >= 2, "nothing was merged"
    bad = {t for t, r in res.items() if r["status"] != 0}
    assert bad == {14, 41}  # the two requests with an id out of range (shifted by the first)
    assert all(res[t]["status"] == P.PLDS_EINVAL for t in bad)
    # replay the logged schedule on the oracle, and apply every request alone on a plain graph
    o, alone = O.OraclePLDS(n), P.PLDS(n)
    t = 0
    while t < len(reqs):
        r = res[t]
        assert r["batch_first"] == t
        group = list(range(t, t + r["batch_size"]))
        assert all(res[u]["batch_first"] == t and res[u]["batch_size"] == len(group) for u in group)
        if kinds[t] == 2:
            assert len(group) == 1
            exp = o.coreness()
            assert np.allclose(outs[t], exp, rtol=1e-12, atol=0), t
            core = O.exact_coreness(n, o.edges())
            assert _within_bound(outs[t], core), f"query {t} in the mix"
            assert _within_bound(alone.coreness(), core), f"query {t} alone"
        else:
            assert all(kinds[u] == kinds[t] for u in group)
            good = [src[u] for u in group if u not in bad]
            batch = np.concatenate(good) if good else np.zeros((0, 2), np.int32)
            assert (o.insert if kinds[t] == 0 else o.delete)(batch) == 0
            st = o.stats()
            for key in ("valid", "rounds", "moves"):
                assert r[key] == st[key], (t, key, r[key], st[key])
            for u in group:
                if u not in bad:
                    (alone.insert if kinds[u] == 0 else alone.delete)(src[u])
        t += len(group)
    assert np.array_equal(served.levels(), o.levels())
    for a, b in zip(served.counters(), o.counters()):
        assert np.array_equal(a, b)
    served.close()
    alone.close()


def test_admission_is_gated_by_memory(P):
    """With the pool limited to its current size, a request whose worst-case growth
    does not fit is refused at submission (nothing admitted, graph unchanged) while a
    deletion and a query still go through."""
    n = 20_000
    e = W.chung_lu(n, 100_000, 2.3, seed=31)
    g = P.PLDS(n)
    g.insert(e[:50_000])
    sv = P.Server(g, slots=4, max_batch=200_000, pool_limit_bytes=1)
    with pytest.raises(P.PldsError) as ex:
        sv.submit(0, edges=e[50_000:])
    assert ex.value.code == P.PLDS_ENOMEM
    sv.submit(1, edges=e[:10])
    out = np.zeros(n)
    sv.submit(2, out=out)
    sv.drain()
    res = sv.poll()
    assert [r["status"] for r in res] == [0, 0]
    sv.close()
    o = O.OraclePLDS(n)
    o.insert(e[:50_000])
    o.delete(e[:10])
    assert np.array_equal(g.levels(), o.levels())
    g.close()
