"""Serving form: requests served by the device-resident loop give the same results
as the same requests applied one call at a time (GPU).

A mixed stream of insertion and deletion batches of uneven sizes (10 .. 20,000
edges, from device, pinned and pageable host buffers) with coreness queries in
between is submitted faster than it is served, so requests wait for ring slots
and run back to back.  Every request's work counts, every query's values, and the
final levels must equal those of a second graph that applies the same requests
with plds_batch_insert / plds_batch_delete / plds_coreness; a dense batch forces the
adjacency pool to grow while the loop runs.
"""
import numpy as np
import pytest

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
    sv = P.Server(served, slots=4, max_batch=400_000)
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
