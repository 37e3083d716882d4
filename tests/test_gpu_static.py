"""Static (2+eps')-approximate k-core (Algorithm 6) on the GPU against the CPU oracle.

Estimates are copies of the same threshold table's doubles on both sides, so they
must be equal exactly, and the iteration counts and neighbour visits must match; the
graph is the handle's current one (after dynamic batches), including isolated
vertices and the paper's worked example.
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


def _same(g, o, ep, what):
    ge, gs = g.static_coreness(ep)
    oe, os_ = o.static_coreness(ep)
    assert np.array_equal(ge, oe), f"{what}: estimates differ at {np.nonzero(ge != oe)[0][:5]}"
    assert gs == os_, f"{what}: {gs} vs {os_}"


def test_static_worked_example(P):
    u, x, y, z, v, w, a, b = range(8)
    E = np.array([(u, x), (u, y), (u, z), (x, y), (x, z), (y, z), (v, u), (v, w), (w, x), (a, y), (a, b),
                  (b, z)], np.int32)
    g = P.PLDS(8)
    g.insert(E)
    est, st = g.static_coreness(4.0)
    assert list(est) == [4, 4, 4, 4, 2, 2, 2, 2]
    g.close()


@pytest.mark.parametrize("ep", [0.5, 1.0, 4.0])
def test_static_matches_oracle(P, ep):
    n = 20_000
    e = W.chung_lu(n, 150_000, 2.2, seed=5)
    g, o = P.PLDS(n), O.OraclePLDS(n)
    for i, bt in enumerate(W.batches(W.shuffled(e, 1), 50_000)):
        g.insert(bt)
        o.insert(bt)
        _same(g, o, ep, f"after insert {i}")
    dl = W.shuffled(e, 2)[:60_000]
    g.delete(dl)
    o.delete(dl)
    _same(g, o, ep, "after delete")
    g.close()


def test_static_rmat_and_device_output(P):
    scale = 15
    n = 1 << scale
    e = W.rmat(scale, 16, seed=7)
    g, o = P.PLDS(n), O.OraclePLDS(n)
    g.insert(e)
    o.insert(e)
    _same(g, o, 2.0, "rmat 15")
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    g.static_coreness(2.0, out=d)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), o.static_coreness(2.0)[0])
    g.close()
