"""The counter-based Chung-Lu draws (CPU): the host (numpy) and torch computations
give the same pairs, any slice equals the same slice of a longer run, and the
endpoint frequencies follow the quantised weights."""
import numpy as np
import pytest

from paper_2106_03824_gb300 import workloads as W

torch = pytest.importorskip("torch")


def test_numpy_and_torch_draws_are_identical():
    g = W.ChungLuDraws(50_000, 400_000, 2.1, seed=3)
    a = g.draws(123_456, 200_000, chunk=1 << 15)
    b = g.draws_torch(123_456, 200_000, device="cpu", chunk=1 << 16).numpy()
    assert np.array_equal(a, b)


def test_slices_are_independent_of_the_run():
    g = W.ChungLuDraws(10_000, 50_000, 2.5, seed=1)
    whole = g.draws(0, 30_000)
    assert np.array_equal(whole[7_000:19_000], g.draws(7_000, 12_000))
    # another seed gives another stream; the same seed the same
    assert not np.array_equal(whole, W.ChungLuDraws(10_000, 50_000, 2.5, seed=2).draws(0, 30_000))
    assert np.array_equal(whole, W.ChungLuDraws(10_000, 50_000, 2.5, seed=1).draws(0, 30_000))


def test_hash_stays_in_range_and_int64_safe():
    x = np.array([0, 1, 2 ** 31 - 2, 2 ** 31 - 1, 2 ** 31, 5 * 10 ** 9, 2 ** 40 + 17], dtype=np.int64)
    h = W._h31(x, 7)
    assert ((h >= 0) & (h < 2 ** 31)).all()
    assert np.array_equal(h, W._h31(torch.from_numpy(x), 7).numpy())
    assert len(set(h.tolist())) == len(h)


def test_endpoint_frequencies_follow_the_weights():
    n = 2_000
    g = W.ChungLuDraws(n, 20_000, 2.2, seed=5)
    d = g.draws(0, 400_000)
    inv = np.empty(n, np.int64)
    inv[g.perm] = np.arange(n)  # back to weight order
    cnt = np.bincount(inv[d.ravel()], minlength=n)
    q = np.diff(np.concatenate([[0], g.cw])).astype(np.float64)
    expect = q / q.sum() * cnt.sum()
    # the heaviest vertices: counts within 5 standard deviations of the expectation
    top = np.argsort(-expect)[:50]
    assert (np.abs(cnt[top] - expect[top]) <= 5 * np.sqrt(expect[top]) + 1).all()
    # and the whole histogram: chi-square per degree of freedom near 1
    chi = ((cnt - expect) ** 2 / np.maximum(expect, 1e-9)).sum() / n
    assert 0.8 < chi < 1.25
    # ids are a permutation of 0..n-1
    assert np.array_equal(np.sort(g.perm), np.arange(n))
