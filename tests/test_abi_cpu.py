"""The C-ABI library builds, loads and exports every entry point of include/plds.h
(CPU only: no compute calls), and the host-side threshold tables agree with the
oracle's (both compute them with their own exact arithmetic)."""
import ctypes

import numpy as np
import pytest

from paper_2106_03824_gb300 import _build
from paper_2106_03824_gb300 import plds as P


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return P.load()


def test_header_declares_the_boundary():
    names = P.exported_symbols_in_header()
    for must in ("plds_create", "plds_batch_insert", "plds_batch_delete", "plds_coreness",
                 "plds_levels", "plds_destroy", "plds_last_status"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in P.exported_symbols_in_header() if not hasattr(lib, s)]
    assert not missing, f"symbols declared in plds.h but not exported: {missing}"


def test_library_has_no_oracle_dependency():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", str(P.LIB_PATH)], capture_output=True, text=True).stdout
    assert "orc_" not in out
    src = "".join(p.read_text() for p in (_build.CSRC).iterdir() if p.is_file())
    assert "oracle" not in src.lower()


def test_invalid_parameters_rejected_without_device(lib):
    # parameter validation happens before any CUDA call
    for args in [(0, 0.4, 3.0), (10, 0.0, 3.0), (10, 0.4, -1.0)]:
        h = lib.plds_create(*args)
        assert not h
        assert lib.plds_last_status() == P.PLDS_EINVAL
    assert lib.plds_batch_insert(None, None, 0) == P.PLDS_EINVAL
    assert lib.plds_levels(None, None) == P.PLDS_EINVAL


def test_serving_admission_rule(lib):
    """The serving loop's admission rule (pure host function): admit when the pool has
    room or a grown pool holding every used and promised slot fits in free memory;
    otherwise wait while earlier requests are in flight, else reject."""
    A = P.server_admission
    assert A(1000, 400, 100, 500, 0) == 0          # room in the pool, exactly
    assert A(1000, 400, 0, 601, 0) == 2            # no room, nothing in flight, no memory
    assert A(1000, 400, 101, 500, 0) == 1          # no room, but requests in flight
    assert A(1000, 400, 100, 501, 4 * 1001) == 0   # a grown pool of 1001 slots fits
    assert A(1000, 400, 100, 501, 4 * 1001 - 1) == 1
    assert A(1000, 400, 0, 601, 4 * 1001 - 1) == 2
    assert A(1000, 1000, 0, 0, 0) == 0             # deletions and queries need nothing
    assert A(-1, 0, 0, 0, 0) == P.PLDS_EINVAL
    assert A(0, 0, 0, 1, -5) == P.PLDS_EINVAL
