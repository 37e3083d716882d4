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
