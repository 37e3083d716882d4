"""Python binding of the GB300 PLDS C ABI (include/plds.h).

Argument marshalling only: every step of a batch runs in the library's CUDA
kernels.  PyTorch supplies device memory (through the caching allocator, when
requested) and the current CUDA stream.  There is no CPU fallback: if the
library cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_lib" / "libplds_gb300.so"

PLDS_OK, PLDS_EINVAL, PLDS_ENOMEM, PLDS_ETIMEOUT, PLDS_EDEVICE, PLDS_EINTERNAL, PLDS_EPOISONED = \
    0, -1, -2, -3, -4, -5, -6
FLAG_HEURISTIC = 1  # Invariant 1's coefficient 2 + 3/lambda replaced by 1.1
FLAG_JUMP = 2  # insertion violators move straight to their targets (the experiments' variant)
_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ETIMEOUT", -4: "EDEVICE", -5: "EINTERNAL",
          -6: "EPOISONED"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class PldsAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class PldsStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "submitted", "self_loops", "duplicates", "filtered", "valid", "rounds", "moves", "visits",
        "dl_evals", "dl_visits", "slots_scanned", "pool_slots_used", "pool_slots_cap", "device_bytes",
        "pool_grows", "err_bits", "err_site")] + [("err_info", ctypes.c_int64 * 3)] + \
        [(k, ctypes.c_int64) for k in ("kernel_ns", "launches", "up_visits", "affected", "skipped_rounds",
                                        "skipped_moves", "skipped_visits", "skipped_up_visits", "pre_ns")]

    def as_dict(self):
        d = {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "err_info"}
        d["err_info"] = [int(x) for x in self.err_info]
        return d


class PldsTuning(ctypes.Structure):
    _fields_ = [("thread_max_cap", ctypes.c_int32), ("load_num", ctypes.c_int32),
                ("load_den", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("test_delay_us", ctypes.c_int32),
                ("trace_rounds", ctypes.c_int32), ("barrier_sleep_ns", ctypes.c_int32),
                ("block_cap", ctypes.c_int32), ("track_orientation", ctypes.c_int32),
                ("list_cap", ctypes.c_int32)]

    KNOBS = ("thread_max_cap", "block_cap", "load_num", "load_den", "list_cap")

    def knobs(self) -> dict:
        return {k: int(getattr(self, k)) for k in self.KNOBS}


TUNE_COST = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.POINTER(PldsTuning), ctypes.c_void_p)


class RequestResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_int64), ("op", ctypes.c_int32), ("status", ctypes.c_int32),
                ("valid", ctypes.c_int64), ("rounds", ctypes.c_int64), ("moves", ctypes.c_int64),
                ("device_ns", ctypes.c_int64), ("batch_first", ctypes.c_int64), ("batch_size", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("done_ns", ctypes.c_int64)]


class PldsError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: PLDS_{_NAMES.get(code, code)} ({code})")
        self.code = code


_lib = None


def load():
    """Load the in-tree CUDA library (build it first with ``_build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise ImportError(f"PLDS CUDA library not built: {LIB_PATH} is missing "
                          "(run __graft_entry__.build())")
    L = ctypes.CDLL(str(LIB_PATH))
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.plds_create.restype = vp
    L.plds_create.argtypes = [i32, dbl, dbl]
    L.plds_create_ex.restype = vp
    L.plds_create_ex.argtypes = [i32, dbl, dbl, i32, ctypes.POINTER(PldsAllocator), vp, ctypes.c_uint32]
    L.plds_batch_insert.argtypes = [vp, vp, i64]
    L.plds_batch_delete.argtypes = [vp, vp, i64]
    L.plds_coreness.argtypes = [vp, vp]
    L.plds_coreness_exponent.argtypes = [vp, vp]
    L.plds_levels.argtypes = [vp, vp]
    L.plds_counters.argtypes = [vp, vp, vp, vp]
    L.plds_stats.argtypes = [vp, ctypes.POINTER(PldsStats)]
    L.plds_params.argtypes = [vp, vp]
    L.plds_tables.argtypes = [vp, vp, vp]
    L.plds_set_stream.argtypes = [vp, vp]
    L.plds_set_tuning.argtypes = [vp, ctypes.POINTER(PldsTuning)]
    L.plds_set_wait_limit.argtypes = [vp, i64]
    L.plds_trace.argtypes = [vp, vp, i32]
    L.plds_set_create.restype = vp
    L.plds_set_create.argtypes = [i32, vp, dbl, dbl, ctypes.POINTER(PldsAllocator), vp]
    L.plds_set_update.argtypes = [vp, vp, vp]
    L.plds_set_graph.restype = vp
    L.plds_set_graph.argtypes = [vp, i32]
    L.plds_set_destroy.argtypes = [vp]
    L.plds_set_destroy.restype = None
    L.plds_set_tune.argtypes = [vp, ctypes.POINTER(PldsTuning)]
    L.plds_set_autotune.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                    i32, i32, ctypes.POINTER(PldsTuning)]
    L.plds_tune_search.argtypes = [ctypes.POINTER(PldsTuning), TUNE_COST, vp, i32, ctypes.POINTER(PldsTuning)]
    L.plds_autotune.argtypes = [vp, vp, vp, vp, i32, i32, i32, ctypes.POINTER(PldsTuning)]
    L.plds_server_create.restype = vp
    L.plds_server_create.argtypes = [vp, i32, i64]
    L.plds_server_submit.argtypes = [vp, i32, vp, i64, vp, ctypes.POINTER(ctypes.c_int64)]
    L.plds_server_poll.argtypes = [vp, ctypes.POINTER(RequestResult), i32]
    L.plds_server_drain.argtypes = [vp]
    L.plds_server_destroy.argtypes = [vp]
    L.plds_server_destroy.restype = None
    L.plds_server_configure.argtypes = [vp, i64, i64]
    L.plds_server_admission.argtypes = [i64, i64, i64, i64, i64]
    L.plds_orient.argtypes = [vp, vp, i64, vp]
    L.plds_out_degrees.argtypes = [vp, vp]
    L.plds_flips.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_int64)]
    L.plds_oriented_updates.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_int64)]
    L.plds_static_coreness.argtypes = [vp, dbl, vp, vp]
    L.plds_opt_levels_per_group.argtypes = [i64, dbl]
    L.plds_opt_levels_per_group.restype = i32
    L.plds_last_status.argtypes = []
    L.plds_destroy.argtypes = [vp]
    L.plds_destroy.restype = None
    _lib = L
    return L


def _ptr(x):
    """Data pointer of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous (np.ascontiguousarray)")
        return ctypes.c_void_p(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError(f"unsupported buffer type {type(x)}")


def _torch_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _torch_allocator():
    """Allocator callbacks backed by PyTorch's CUDA caching allocator."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or 0)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a = PldsAllocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    return a


class PLDS:
    """One graph on the current CUDA device; wraps a plds_t handle."""

    def __init__(self, n: int, delta: float = 0.4, lam: float = 3.0, levels_per_group: int = 0,
                 torch_allocator: bool = True, stream=None, _borrowed=None, heuristic: bool = False,
                 jump: bool = False):
        L = load()
        self.n = int(n)
        self._owned = _borrowed is None
        if _borrowed is not None:  # a graph owned by a PLDSSet
            self._alloc = None
            self._h = _borrowed
        else:
            self._alloc = _torch_allocator() if torch_allocator else None
            st = stream if stream is not None else (_torch_stream() if torch_allocator else None)
            self._h = L.plds_create_ex(self.n, float(delta), float(lam), int(levels_per_group),
                                       ctypes.byref(self._alloc) if self._alloc else None, st,
                                       (FLAG_HEURISTIC if heuristic else 0) | (FLAG_JUMP if jump else 0))
        if not self._h:
            raise PldsError(L.plds_last_status(), "plds_create_ex")
        p = np.zeros(4, np.int32)
        L.plds_params(self._h, _ptr(p))
        self.t, self.Lg, self.G, self.K = (int(x) for x in p)

    def _check(self, rc, what):
        if rc != PLDS_OK:
            raise PldsError(rc, what)

    def close(self):
        if getattr(self, "_h", None):
            if self._owned:
                load().plds_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- batches ---------------------------------------------------------
    @staticmethod
    def _edges(edges):
        if isinstance(edges, np.ndarray):
            return np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
        if edges.dtype != __import__("torch").int32 or not edges.is_contiguous():
            raise ValueError("edge tensor must be contiguous int32 [B,2]")
        return edges

    def insert(self, edges, check=True) -> int:
        """edges: int32 [B,2] numpy array (host) or torch tensor (host or cuda)."""
        edges = self._edges(edges)
        rc = load().plds_batch_insert(self._h, _ptr(edges), int(edges.shape[0]))
        if check:
            self._check(rc, "plds_batch_insert")
        return rc

    def delete(self, edges, check=True) -> int:
        edges = self._edges(edges)
        rc = load().plds_batch_delete(self._h, _ptr(edges), int(edges.shape[0]))
        if check:
            self._check(rc, "plds_batch_delete")
        return rc

    # -- queries ---------------------------------------------------------
    def coreness(self, out=None):
        out = np.zeros(self.n, np.float64) if out is None else out
        self._check(load().plds_coreness(self._h, _ptr(out)), "plds_coreness")
        return out

    def coreness_exponent(self, out=None):
        out = np.zeros(self.n, np.int32) if out is None else out
        self._check(load().plds_coreness_exponent(self._h, _ptr(out)), "plds_coreness_exponent")
        return out

    def levels(self, out=None):
        out = np.zeros(self.n, np.int32) if out is None else out
        self._check(load().plds_levels(self._h, _ptr(out)), "plds_levels")
        return out

    def counters(self, out=None):
        """(deg, up, up*); out = three preallocated int32 buffers (host or device) or None."""
        d, u, s = out if out is not None else (np.zeros(self.n, np.int32) for _ in range(3))
        self._check(load().plds_counters(self._h, _ptr(d), _ptr(u), _ptr(s)), "plds_counters")
        return d, u, s

    def stats(self) -> dict:
        st = PldsStats()
        self._check(load().plds_stats(self._h, ctypes.byref(st)), "plds_stats")
        return st.as_dict()

    def tables(self):
        up = np.zeros(self.G, np.int32)
        dn = np.zeros(self.G, np.int32)
        self._check(load().plds_tables(self._h, _ptr(up), _ptr(dn)), "plds_tables")
        return up, dn

    def set_tuning(self, **kw):
        t = PldsTuning()
        for k, v in kw.items():
            setattr(t, k, int(v))
        self._check(load().plds_set_tuning(self._h, ctypes.byref(t)), "plds_set_tuning")

    def autotune(self, batches, timed_from: int = 1, max_trials: int = 12) -> dict:
        """Pick this handle's speed-only knobs on a sample stream applied to scratch
        handles built alike: batches = [(kind, edges)] with kind "ins" or "del" and
        edges int32 [B, 2] (host arrays, or device tensors for representative
        timings), the ones before timed_from untimed.  The graph is not touched;
        the best knobs are applied and returned."""
        edges = [self._edges(e) for _, e in batches]
        offs = np.zeros(len(edges) + 1, np.int64)
        offs[1:] = np.cumsum([e.shape[0] for e in edges])
        kinds = np.array([0 if k == "ins" else 1 for k, _ in batches], np.int32)
        if all(isinstance(e, np.ndarray) for e in edges):
            flat = np.ascontiguousarray(np.concatenate(edges) if edges else np.zeros((0, 2), np.int32))
        else:
            torch = __import__("torch")
            flat = torch.cat([torch.as_tensor(e).to(edges[0].device) for e in edges]).contiguous()
        best = PldsTuning()
        rc = load().plds_autotune(self._h, _ptr(flat), _ptr(offs), _ptr(kinds), len(edges), int(timed_from),
                                  int(max_trials), ctypes.byref(best))
        self._check(rc, "plds_autotune")
        return best.knobs()

    def static_coreness(self, eps_prime: float = 1.0, out=None):
        """Static (2+eps')-approximate k-core of the current graph (Algorithm 6):
        (estimates, {outer, inner, visits})."""
        out = np.zeros(self.n, np.float64) if out is None else out
        st = np.zeros(3, np.int64)
        self._check(load().plds_static_coreness(self._h, float(eps_prime), _ptr(out), _ptr(st)),
                    "plds_static_coreness")
        return out, dict(outer=int(st[0]), inner=int(st[1]), visits=int(st[2]))

    # orientation (Algorithm 5)
    def orient(self, edges) -> np.ndarray:
        """Tail (source endpoint) of each edge, -1 if absent or invalid."""
        e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2) if isinstance(edges, np.ndarray) \
            else edges
        out = np.zeros(e.shape[0], np.int32)
        self._check(load().plds_orient(self._h, _ptr(e), int(e.shape[0]), _ptr(out)), "plds_orient")
        return out

    def out_degrees(self) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        self._check(load().plds_out_degrees(self._h, _ptr(out)), "plds_out_degrees")
        return out

    def _pairs(self, fn, name) -> np.ndarray:
        cnt = ctypes.c_int64()
        self._check(fn(self._h, None, 0, ctypes.byref(cnt)), name)
        out = np.zeros((max(cnt.value, 1), 2), np.int32)
        self._check(fn(self._h, _ptr(out), cnt.value, ctypes.byref(cnt)), name)
        return out[:cnt.value]

    def flips(self) -> np.ndarray:
        """F of the last tracked batch call: (tail, head) before the flip, unordered."""
        return self._pairs(load().plds_flips, "plds_flips")

    def oriented_updates(self) -> np.ndarray:
        """J of the last tracked batch call, unordered."""
        return self._pairs(load().plds_oriented_updates, "plds_oriented_updates")

    def trace(self, cap: int = 1 << 16):
        out = np.zeros((cap, 12), np.int32)
        k = load().plds_trace(self._h, _ptr(out), cap)
        if k < 0:
            raise PldsError(k, "plds_trace")
        return out[:k]

    def set_wait_limit(self, ns: int):
        self._check(load().plds_set_wait_limit(self._h, int(ns)), "plds_set_wait_limit")

    def set_stream(self, stream):
        self._check(load().plds_set_stream(self._h, stream), "plds_set_stream")


class PLDSSet:
    """Independent graphs updated together, one kernel launch per round (batched form)."""

    def __init__(self, ns, delta: float = 0.4, lam: float = 3.0, torch_allocator: bool = True):
        L = load()
        self.ns = [int(x) for x in ns]
        arr = np.asarray(self.ns, np.int32)
        self._alloc = _torch_allocator() if torch_allocator else None
        st = _torch_stream() if torch_allocator else None
        self._s = L.plds_set_create(len(self.ns), _ptr(arr), float(delta), float(lam),
                                    ctypes.byref(self._alloc) if self._alloc else None, st)
        if not self._s:
            raise PldsError(L.plds_last_status(), "plds_set_create")
        self.graphs = [PLDS(n, _borrowed=L.plds_set_graph(self._s, i)) for i, n in enumerate(self.ns)]

    def update(self, edges, offsets, check=True) -> int:
        """edges: int32 [total,2] (host array or cuda tensor); offsets: int64 [2*count+1]."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        if isinstance(edges, np.ndarray):
            edges = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
        rc = load().plds_set_update(self._s, _ptr(edges), _ptr(off))
        if check and rc != PLDS_OK:
            raise PldsError(rc, "plds_set_update")
        return rc

    def tune(self, **knobs):
        """Apply thread_max_cap / block_cap / load_num / load_den / list_cap to every graph."""
        t = PldsTuning()
        for k, v in knobs.items():
            setattr(t, k, int(v))
        rc = load().plds_set_tune(self._s, ctypes.byref(t))
        if rc != PLDS_OK:
            raise PldsError(rc, "plds_set_tune")

    def autotune(self, rounds, timed_from: int = 0, max_trials: int = 24) -> dict:
        """Pick the knobs on a sample of the workload: rounds = [(edges, offsets)]
        (as for update; device tensors give representative timings), the ones before
        timed_from untimed.  Applies the best knobs and returns them."""
        keep = []
        ep = (ctypes.c_void_p * len(rounds))()
        op = (ctypes.c_void_p * len(rounds))()
        for r, (e, o) in enumerate(rounds):
            if isinstance(e, np.ndarray):
                e = np.ascontiguousarray(e, dtype=np.int32).reshape(-1, 2)
            o = np.ascontiguousarray(o, dtype=np.int64)
            keep.append((e, o))
            ep[r] = _ptr(e).value
            op[r] = _ptr(o).value
        best = PldsTuning()
        rc = load().plds_set_autotune(self._s, len(rounds), ep, op, int(timed_from), int(max_trials),
                                      ctypes.byref(best))
        if rc != PLDS_OK:
            raise PldsError(rc, "plds_set_autotune")
        return best.knobs()

    @staticmethod
    def pack(halves):
        """[(ins_i, del_i)] per graph -> (edges [total,2], offsets [2*count+1])."""
        parts, offs, pos = [], [0], 0
        for ins, dele in halves:
            for h in (ins, dele):
                h = np.asarray(h, np.int32).reshape(-1, 2)
                parts.append(h)
                pos += h.shape[0]
                offs.append(pos)
        edges = np.ascontiguousarray(np.concatenate(parts)) if parts else np.zeros((0, 2), np.int32)
        return edges, np.asarray(offs, np.int64)

    def close(self):
        if getattr(self, "_s", None):
            for g in self.graphs:
                g._h = None
            load().plds_set_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Device-resident request loop over one PLDS graph (serving form)."""
    INSERT, DELETE, CORENESS = 0, 1, 2

    def __init__(self, graph: "PLDS", slots: int = 8, max_batch: int = 1 << 20, merge_max_edges: int = -1,
                 pool_limit_bytes: int = 0):
        """merge_max_edges: edges one merged batch may hold (0 = every request is its
        own batch, -1 = max_batch); pool_limit_bytes: cap on the adjacency pool
        (0 = free device memory only)."""
        self.g = graph
        self._sv = load().plds_server_create(graph._h, int(slots), int(max_batch))
        if not self._sv:
            raise PldsError(load().plds_last_status(), "plds_server_create")
        self._keep = {}  # buffers that must stay alive until their request finishes
        self.configure(merge_max_edges, pool_limit_bytes)

    def configure(self, merge_max_edges: int = -1, pool_limit_bytes: int = 0):
        rc = load().plds_server_configure(self._sv, int(merge_max_edges), int(pool_limit_bytes))
        if rc != PLDS_OK:
            raise PldsError(rc, "plds_server_configure")

    def submit(self, op: int, edges=None, out=None) -> int:
        t = ctypes.c_int64()
        if op == self.CORENESS:
            rc = load().plds_server_submit(self._sv, op, None, 0, _ptr(out), ctypes.byref(t))
        else:
            if isinstance(edges, np.ndarray):
                edges = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
            elif getattr(edges, "is_cuda", False):
                # the loop reads device buffers in place: their producing work must be done
                __import__("torch").cuda.current_stream().synchronize()
            rc = load().plds_server_submit(self._sv, op, _ptr(edges), int(edges.shape[0]), None,
                                           ctypes.byref(t))
        if rc != PLDS_OK:
            raise PldsError(rc, "plds_server_submit")
        self._keep[t.value] = (edges, out)
        return t.value

    def poll(self, cap: int = 1024):
        buf = (RequestResult * cap)()
        k = load().plds_server_poll(self._sv, buf, cap)
        if k < 0:
            raise PldsError(k, "plds_server_poll")
        res = [dict(ticket=r.ticket, op=r.op, status=r.status, valid=r.valid, rounds=r.rounds,
                    moves=r.moves, device_ns=r.device_ns, batch_first=r.batch_first,
                    batch_size=r.batch_size, done_ns=r.done_ns) for r in buf[:k]]
        for r in res:
            self._keep.pop(r["ticket"], None)
        return res

    def drain(self):
        rc = load().plds_server_drain(self._sv)
        if rc != PLDS_OK:
            raise PldsError(rc, "plds_server_drain")

    def close(self):
        if getattr(self, "_sv", None):
            load().plds_server_destroy(self._sv)
            self._sv = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_search(cost, start: dict | None = None, max_trials: int = 24):
    """The autotuner's coordinate descent against a Python cost function
    cost(knobs: dict) -> float (no device use).  Returns (best knobs, evaluations)."""
    st = PldsTuning()
    for k, v in (start or {}).items():
        setattr(st, k, int(v))

    def _cb(t, _ctx):
        try:
            return float(cost(t.contents.knobs()))
        except Exception:
            return -1.0

    cb = TUNE_COST(_cb)
    best = PldsTuning()
    k = load().plds_tune_search(ctypes.byref(st), cb, None, int(max_trials), ctypes.byref(best))
    if k < 0:
        raise PldsError(k, "plds_tune_search")
    return best.knobs(), k


def opt_levels_per_group(m: int, delta: float = 0.4) -> int:
    """Levels per group of PLDSOpt for a graph of about m edges (pass it as
    levels_per_group); raises on invalid input."""
    r = load().plds_opt_levels_per_group(int(m), float(delta))
    if r < 0:
        raise PldsError(r, "plds_opt_levels_per_group")
    return r


def server_admission(pool_cap: int, pool_used: int, inflight: int, need: int, free_bytes: int) -> int:
    """The serving loop's admission rule (no device use): 0 admit, 1 wait, 2 reject."""
    return load().plds_server_admission(int(pool_cap), int(pool_used), int(inflight), int(need),
                                        int(free_bytes))


def exported_symbols_in_header(header: os.PathLike | None = None):
    """Function names declared in include/plds.h."""
    import re
    header = Path(header) if header else _PKG.parent / "include" / "plds.h"
    text = header.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(plds_[a-z_]+)\s*\(", text)))
