"""Algorithmic-byte definitions of bench.py's roofline (CPU): executed work only
(skipped rounds left out), the scope table's per-unit figures, and the
Algorithm-2-equivalent count with the skipped rounds."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

S = {"submitted": 1000, "valid": 900, "moves": 500, "skipped_moves": 300, "visits": 7000,
     "skipped_visits": 4000, "up_visits": 3000, "skipped_up_visits": 1800, "affected": 250, "dl_visits": 60}


def test_executed_bytes_insertion():
    # 8*1000 + 64*900 + 4*(500-300) + 8*(3000-1800) + 8*60
    assert bench.algo_bytes(S, "ins") == 8000 + 57600 + 800 + 9600 + 480


def test_executed_bytes_deletion_uses_degrees():
    assert bench.algo_bytes(S, "del") == 8000 + 57600 + 800 + 8 * 3000 + 480


def test_degree_definition():
    # per move its degree and its affected neighbours: 8*(7000-4000) + 8*250
    assert bench.algo_bytes_degree(S) == 8000 + 57600 + 800 + 24000 + 2000 + 480


def test_with_skipped_rounds():
    assert bench.algo_bytes_with_skipped(S, "ins") == 8000 + 57600 + 2000 + 24000 + 480
    z = dict(S, skipped_moves=0, skipped_visits=0, skipped_up_visits=0)
    assert bench.algo_bytes_with_skipped(z, "ins") == bench.algo_bytes(z, "ins")


def test_step_bytes_are_part_of_executed_bytes():
    # the step kernels' share: 8 per submitted edge + 64 per applied update
    assert bench.algo_bytes_steps(S) == 8000 + 57600
    for kind in ("ins", "del"):
        assert bench.algo_bytes(S, kind) - bench.algo_bytes_steps(S) > 0


def test_unique_edges_of_a_raw_pair_stream():
    """The large form's distinct-edge set of raw draws (CPU tensors here): self-loops
    dropped, (u, v) and (v, u) one edge, canonical u < v, sorted by key."""
    torch = __import__("pytest").importorskip("torch")
    pairs = torch.tensor([[3, 1], [1, 3], [2, 2], [0, 5], [5, 0], [4, 1], [1, 4], [6, 7]], dtype=torch.int32)
    out = bench.unique_edges_device(pairs)
    assert out.dtype == torch.int32
    assert out.tolist() == [[0, 5], [1, 3], [1, 4], [6, 7]]


def test_sha_of_int32_arrays_is_little_endian_concatenation():
    import hashlib
    import numpy as np
    a, b = np.array([1, -2], np.int32), np.array([7], np.int64)
    want = hashlib.sha256(np.array([1, -2, 7], "<i4").tobytes()).hexdigest()
    assert bench.sha_i32(a, b) == want
