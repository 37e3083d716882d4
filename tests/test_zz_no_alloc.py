"""plds_batch_static: the allocation-free batch call (GPU).

Callers that must not allocate device memory during updates (latency-critical
loops, fixed memory budgets) use plds_batch_static, whose per-batch scratch lives
in one library-wide device array.  This checks, through the C ABI, that two calls
in a row give the same levels and coreness as the regular entry points on an
identical graph.  Kept in a file that runs last so a failure here leaves the other
GPU tests already run.
"""
import ctypes

import numpy as np
import pytest

from paper_2106_03824_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-12


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2106_03824_gb300 import plds
    L = plds.load()
    L.plds_batch_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]
    L.plds_batch_static.restype = ctypes.c_int
    return plds


def _static(P, g, edges, is_delete):
    e = np.ascontiguousarray(edges, dtype=np.int32)
    return P.load().plds_batch_static(g._h, ctypes.c_void_p(e.ctypes.data), e.shape[0], is_delete)


def test_static_batches_match_regular_calls(P):
    n = 6000
    e = W.chung_lu(n, 40_000, 2.3, seed=21)
    ins = W.shuffled(e, 5)
    a = P.PLDS(n)
    b = P.PLDS(n)
    # two insertion calls in a row, then two deletion calls in a row
    for k, batch in enumerate((ins[:30_000], ins[30_000:])):
        a.insert(batch)
        assert _static(P, b, batch, 0) == P.PLDS_OK
        assert np.array_equal(a.levels(), b.levels()), f"insert call {k}"
        assert np.allclose(a.coreness(), b.coreness(), rtol=REL_TOL, atol=0)
        assert a.stats()["moves"] == b.stats()["moves"]
    dele = W.shuffled(e, 6)
    for k, batch in enumerate((dele[:20_000], dele[20_000:35_000])):
        a.delete(torch.from_numpy(batch).cuda())
        assert _static(P, b, batch, 1) == P.PLDS_OK
        assert np.array_equal(a.levels(), b.levels()), f"delete call {k}"
        assert np.allclose(a.coreness(), b.coreness(), rtol=REL_TOL, atol=0)
    a.close()
    b.close()


def test_static_rejects_oversized_batches(P):
    g = P.PLDS(100)
    big = np.zeros((65_537, 2), np.int32)
    assert _static(P, g, big, 0) == P.PLDS_EINVAL
    assert _static(P, g, big[:10], 2) == P.PLDS_EINVAL
    g.close()


def test_static_rejected_ids_leave_no_trace(P):
    """A static insertion batch with an id outside [0, n) among new valid edges is
    rejected; the next static batches grow the tables and give the results of a
    handle that never saw it."""
    n = 3000
    e = W.erdos_renyi(n, 20_000, seed=43)
    a, b = P.PLDS(n), P.PLDS(n)
    for h in (a, b):
        assert _static(P, h, e[:8000], 0) == P.PLDS_OK
    bad = np.concatenate([e[8000:14000], np.array([[7, n]], np.int32)])
    assert _static(P, a, bad, 0) == P.PLDS_EINVAL
    for h in (a, b):
        assert _static(P, h, e[8000:], 0) == P.PLDS_OK
    assert np.array_equal(a.levels(), b.levels())
    for x, y in zip(a.counters(), b.counters()):
        assert np.array_equal(x, y)
    assert a.stats()["pool_slots_used"] == b.stats()["pool_slots_used"]
    a.close()
    b.close()


def _counting_handle(P, n):
    """A handle whose device memory comes from a counting allocator callback."""
    L = P.load()
    calls = {"alloc": 0, "free": 0}

    def _alloc(nbytes, stream, ctx):
        calls["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)

    def _free(ptr, nbytes, stream, ctx):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    alloc = P.PldsAllocator(P.ALLOC_FN(_alloc), P.FREE_FN(_free), None)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    h = L.plds_create_ex(n, 0.4, 3.0, 0, ctypes.byref(alloc), stream, 0)
    assert h
    return P.PLDS(n, _borrowed=h), h, calls, alloc


def test_static_calls_make_no_allocation(P):
    """Every device buffer the handle owns comes from the caller's allocator; the
    static calls (insertions and deletions, host and device edges) call it zero
    times, and their results equal the regular calls'."""
    n = 5000
    e = W.chung_lu(n, 30_000, 2.3, seed=23)
    g, h, calls, _keep = _counting_handle(P, n)
    ref = P.PLDS(n)
    before = dict(calls)
    ins = W.shuffled(e, 7)
    for batch in (ins[:12_000], ins[12_000:24_000]):
        ref.insert(batch)
        assert _static(P, g, batch, 0) == P.PLDS_OK
    dev = torch.from_numpy(W.shuffled(e, 8)[:9_000]).cuda()  # edges already on the device
    ref.delete(dev)
    rc = P.load().plds_batch_static(h, ctypes.c_void_p(dev.data_ptr()), dev.shape[0], 1)
    assert rc == P.PLDS_OK
    assert calls == before, f"static calls allocated: {calls} vs {before}"
    assert np.array_equal(g.levels(), ref.levels())
    d, u, s = g.counters()
    rd, ru, rs = ref.counters()
    assert np.array_equal(d, rd) and np.array_equal(u, ru) and np.array_equal(s, rs)
    P.load().plds_destroy(h)
    ref.close()


def test_static_full_pool_reports_enomem_unchanged(P):
    """A batch whose tables do not fit the adjacency pool: PLDS_ENOMEM with levels and
    counters as before the call (growing the pool would allocate); a regular call
    with the same batch then grows the pool and gives the oracle's result."""
    from oracle import oracle as O
    n = 2000
    e = W.erdos_renyi(n, 400_000, seed=31)  # ~8 * 400k slots of tables: more than the initial pool
    g, h, calls, _keep = _counting_handle(P, n)
    o = O.OraclePLDS(n)
    hit = False
    for s0 in range(0, e.shape[0], 50_000):
        b = np.ascontiguousarray(e[s0:s0 + 50_000])
        lv, cn = g.levels().copy(), [x.copy() for x in g.counters()]
        before = dict(calls)
        rc = _static(P, g, b, 0)
        assert calls == before
        if rc == P.PLDS_ENOMEM:
            hit = True
            assert np.array_equal(g.levels(), lv)
            for x, y in zip(g.counters(), cn):
                assert np.array_equal(x, y)
            g.insert(b)  # the regular call grows the pool
        else:
            assert rc == P.PLDS_OK
        assert o.insert(b) == 0
        assert np.array_equal(g.levels(), o.levels())
        if hit:
            break
    assert hit, "the pool never filled"
    P.load().plds_destroy(h)
