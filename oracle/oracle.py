"""ctypes wrapper of the sequential CPU PLDS oracle (plds_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU-baseline leg may load this module; the product path never does.  It imports
nothing from the CUDA package.

Every function here marshals arguments only; the arithmetic lives in the C file,
which cites the paper section it follows for each step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "plds_oracle.c"
_OUT = _HERE / "_build" / "libplds_oracle.so"

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_EINTERNAL = 0, -1, -2, -5

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain C11, -O2); returns the .so path."""
    _OUT.parent.mkdir(parents=True, exist_ok=True)
    if force or not _OUT.exists() or _OUT.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _OUT.with_suffix(f".{os.getpid()}.tmp.so")
        # no fused multiply-add contraction: the static k-core's double thresholds must
        # round the same way on every host
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-Wall", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        # PLDS_ORACLE_SO points the tests at a deliberately broken copy of the
        # oracle (mutation tests of the pins); normally the source is built here.
        alt = os.environ.get("PLDS_ORACLE_SO")
        path = Path(alt) if alt else build()
        L = ctypes.CDLL(str(path))
        P = ctypes.c_void_p
        i32p = ctypes.POINTER(ctypes.c_int32)
        L.orc_create.restype = P
        L.orc_create.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32]
        L.orc_create_ex.restype = P
        L.orc_create_ex.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                    ctypes.c_int32]
        L.orc_destroy.argtypes = [P]
        for name in ("orc_insert", "orc_delete", "orc_add_edges_raw"):
            getattr(L, name).argtypes = [P, P, ctypes.c_int64]
        L.orc_update.argtypes = [P, P, ctypes.c_int64, P, ctypes.c_int64]
        for name in ("orc_levels", "orc_coreness", "orc_coreness_exponent", "orc_stats",
                     "orc_params", "orc_edges", "orc_num_edges"):
            getattr(L, name).argtypes = [P, P]
        L.orc_counters.argtypes = [P, P, P, P]
        L.orc_check.argtypes = [P]
        L.orc_set_level.argtypes = [P, ctypes.c_int32, ctypes.c_int32]
        L.orc_tables_query.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                       ctypes.c_int32, i32p, i32p, i32p, i32p, P, P,
                                       ctypes.c_int32]
        L.orc_exact_coreness.argtypes = [ctypes.c_int32, P, ctypes.c_int64, P]
        L.orc_track.argtypes = [P, ctypes.c_int]
        L.orc_orient.argtypes = [P, P, ctypes.c_int64, P]
        L.orc_out_degrees.argtypes = [P, P]
        for name in ("orc_flips", "orc_oriented_updates"):
            getattr(L, name).argtypes = [P, P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        L.orc_opt_levels_per_group.argtypes = [ctypes.c_int64, ctypes.c_double]
        L.orc_static_coreness.argtypes = [P, ctypes.c_double, P, P]
        L.orc_static_thresholds.argtypes = [ctypes.c_int32, ctypes.c_double, P, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_int32)]
        L.orc_static_thresholds.restype = ctypes.c_int32
        L.orc_opt_levels_per_group.restype = ctypes.c_int32
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _edges(e) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(e, dtype=np.int32).reshape(-1, 2))
    return a


def opt_levels_per_group(m: int, delta: float = 0.4) -> int:
    """PLDSOpt's ceil(log_{1+delta}(m) / 50) levels per group (at least 1), exact."""
    r = lib().orc_opt_levels_per_group(int(m), float(delta))
    if r < 0:
        raise ValueError(f"orc_opt_levels_per_group({m}, {delta}) = {r}")
    return r


HEURISTIC = 1  # Invariant 1's coefficient 2 + 3/lambda replaced by 1.1
JUMP = 2  # insertion violators move straight to their targets (the experiments' variant)


def tables(n: int, delta: float = 0.4, lam: float = 3.0, levels_per_group: int = 0, flags: int = 0):
    """Exact (t, Lg, G, K, upmax[G], dnmin[G]) from the oracle's rational arithmetic."""
    L = lib()
    t, Lg, G, K = (ctypes.c_int32() for _ in range(4))
    cap = 8192
    up = np.zeros(cap, np.int32)
    dn = np.zeros(cap, np.int32)
    rc = L.orc_tables_query(n, delta, lam, levels_per_group, flags, ctypes.byref(t), ctypes.byref(Lg),
                            ctypes.byref(G), ctypes.byref(K), _ptr(up), _ptr(dn), cap)
    if rc != ORC_OK:
        raise ValueError(f"orc_tables_query rc={rc}")
    g = G.value
    return dict(t=t.value, Lg=Lg.value, G=g, K=K.value, upmax=up[:g].copy(), dnmin=dn[:g].copy())


def exact_coreness(n: int, edges) -> np.ndarray:
    """Exact coreness of every vertex (Matula-Beck peeling)."""
    e = _edges(edges)
    out = np.zeros(n, np.int32)
    rc = lib().orc_exact_coreness(n, _ptr(e), e.shape[0], _ptr(out))
    if rc != ORC_OK:
        raise ValueError(f"orc_exact_coreness rc={rc}")
    return out


STAT_KEYS = ("submitted", "self_loops", "duplicates", "filtered", "valid", "rounds", "moves",
             "visits", "dl_evals", "dl_visits", "max_vertex_moves", "dir_error")


class OraclePLDS:
    """Sequential PLDS; one instance per graph."""

    def __init__(self, n: int, delta: float = 0.4, lam: float = 3.0, levels_per_group: int = 0,
                 flags: int = 0):
        self.n = n
        self._h = lib().orc_create_ex(n, delta, lam, levels_per_group, flags)
        if not self._h:
            raise ValueError("orc_create failed (bad n / delta / lambda)")
        p = np.zeros(4, np.int32)
        lib().orc_params(self._h, _ptr(p))
        self.t, self.Lg, self.G, self.K = (int(x) for x in p)

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def insert(self, edges) -> int:
        e = _edges(edges)
        return lib().orc_insert(self._h, _ptr(e), e.shape[0])

    def delete(self, edges) -> int:
        e = _edges(edges)
        return lib().orc_delete(self._h, _ptr(e), e.shape[0])

    def add_edges_raw(self, edges) -> int:
        e = _edges(edges)
        return lib().orc_add_edges_raw(self._h, _ptr(e), e.shape[0])

    def set_level(self, v: int, level: int) -> int:
        return lib().orc_set_level(self._h, v, level)

    def levels(self) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        lib().orc_levels(self._h, _ptr(out))
        return out

    def coreness(self) -> np.ndarray:
        out = np.zeros(self.n, np.float64)
        lib().orc_coreness(self._h, _ptr(out))
        return out

    def coreness_exponent(self) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        lib().orc_coreness_exponent(self._h, _ptr(out))
        return out

    def counters(self):
        d = np.zeros(self.n, np.int32)
        u = np.zeros(self.n, np.int32)
        s = np.zeros(self.n, np.int32)
        lib().orc_counters(self._h, _ptr(d), _ptr(u), _ptr(s))
        return d, u, s

    def check(self) -> int:
        return lib().orc_check(self._h)

    def stats(self) -> dict:
        a = np.zeros(12, np.int64)
        lib().orc_stats(self._h, _ptr(a))
        return dict(zip(STAT_KEYS, (int(x) for x in a)))

    def edges(self) -> np.ndarray:
        m = ctypes.c_int64()
        lib().orc_num_edges(self._h, ctypes.byref(m))
        out = np.zeros((m.value, 2), np.int32)
        lib().orc_edges(self._h, _ptr(out))
        return out

    # orientation (Algorithm 5)
    def track(self, on: bool = True):
        lib().orc_track(self._h, 1 if on else 0)

    def orient(self, edges) -> np.ndarray:
        e = _edges(edges)
        out = np.zeros(e.shape[0], np.int32)
        lib().orc_orient(self._h, _ptr(e), e.shape[0], _ptr(out))
        return out

    def out_degrees(self) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        lib().orc_out_degrees(self._h, _ptr(out))
        return out

    def _pairs(self, fn) -> np.ndarray:
        cnt = ctypes.c_int64()
        rc = fn(self._h, None, 0, ctypes.byref(cnt))
        if rc != ORC_OK:
            raise ValueError(f"rc={rc} (tracking off?)")
        out = np.zeros((max(cnt.value, 1), 2), np.int32)
        fn(self._h, _ptr(out), cnt.value, ctypes.byref(cnt))
        return out[:cnt.value]

    def flips(self) -> np.ndarray:
        """Edges of the last batch whose orientation flipped, (tail, head) before, sorted."""
        return self._pairs(lib().orc_flips)

    def oriented_updates(self) -> np.ndarray:
        """The last batch's valid updates oriented as Algorithm 5 returns them, sorted."""
        return self._pairs(lib().orc_oriented_updates)

    # static (2+eps')-approximate k-core (Algorithm 6)
    def static_coreness(self, eps_prime: float = 1.0):
        """(estimates, {outer, inner, visits}) of Algorithm 6 on the current graph."""
        est = np.zeros(self.n, np.float64)
        st = np.zeros(3, np.int64)
        rc = lib().orc_static_coreness(self._h, float(eps_prime), _ptr(est), _ptr(st))
        if rc != ORC_OK:
            raise ValueError(f"orc_static_coreness rc={rc}")
        return est, dict(outer=int(st[0]), inner=int(st[1]), visits=int(st[2]))


def static_thresholds(n: int, eps_prime: float = 1.0):
    """(thresholds (1+eps)^b, J) of Algorithm 6 for n vertices."""
    thr = np.zeros(4096, np.float64)
    J = ctypes.c_int32()
    k = lib().orc_static_thresholds(int(n), float(eps_prime), _ptr(thr), 4096, ctypes.byref(J))
    if k < 0:
        raise ValueError(f"orc_static_thresholds rc={k}")
    return thr[:k].copy(), J.value
