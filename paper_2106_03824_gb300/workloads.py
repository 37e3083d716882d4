"""Seeded synthetic graph workloads and batch streams.

This module only draws random inputs: it holds none of the PLDS arithmetic, so
both the CPU oracle (tests) and the CUDA path (tests, bench) consume the same
arrays.  Every generator is deterministic for a given seed (numpy PCG64).

Graph shapes follow the workloads the paper measures (Section "Experiments":
dataset table and the Ins/Del/Mix protocol): the paper's SNAP/DIMACS graphs are
not available, so these generators stand in with the same sizes and degree
distribution shapes.

All edge arrays are ``int32[m, 2]`` in canonical form (u < v), self-loops and
duplicates removed, vertex ids randomly permuted.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _sorted_unique(keys: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + adjacent compare)."""
    k = np.sort(keys, kind="stable")
    if k.size == 0:
        return k
    keep = np.empty(k.size, dtype=bool)
    keep[0] = True
    np.not_equal(k[1:], k[:-1], out=keep[1:])
    return k[keep]


def _canonical_unique(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Drop self-loops, orient u<v, drop duplicates; returns int32[m,2] sorted by key."""
    u = u.astype(np.int64, copy=False)
    v = v.astype(np.int64, copy=False)
    keep = u != v
    u, v = u[keep], v[keep]
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    key = _sorted_unique((lo << 32) | hi)
    out = np.empty((key.size, 2), dtype=np.int32)
    out[:, 0] = (key >> 32).astype(np.int32)
    out[:, 1] = (key & 0xFFFFFFFF).astype(np.int32)
    return out


def _relabel(edges: np.ndarray, n: int, rng: np.random.Generator) -> np.ndarray:
    perm = rng.permutation(n).astype(np.int32)
    e = perm[edges]
    lo = np.minimum(e[:, 0], e[:, 1])
    hi = np.maximum(e[:, 0], e[:, 1])
    return np.stack([lo, hi], axis=1).astype(np.int32)


def chung_lu(n: int, m: int, gamma: float, seed: int = 1) -> np.ndarray:
    """Chung-Lu power-law graph with ~m unique undirected edges.

    Expected degrees d_i proportional to (i+1)^(-1/(gamma-1)), scaled to mean
    2m/n and truncated at sqrt(2m) (the Chung-Lu validity condition).  Endpoints
    are drawn i.i.d. proportional to d until m unique non-loop edges exist or 4m
    pairs have been drawn.  Vertex ids are randomly permuted.
    """
    rng = _rng(seed)
    if n < 2 or m <= 0:
        return np.zeros((0, 2), dtype=np.int32)
    w = (np.arange(1, n + 1, dtype=np.float64)) ** (-1.0 / (gamma - 1.0))
    cap = np.sqrt(2.0 * m)
    for _ in range(8):  # rescale to the target sum after truncation
        w = w * (2.0 * m / w.sum())
        w = np.minimum(w, cap)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    keys = np.zeros(0, dtype=np.int64)
    drawn = 0
    while keys.size < m and drawn < 4 * m:
        # draw enough for the remaining edges at the duplicate rate seen so far
        rate = drawn / max(keys.size, 1) if drawn else 1.2
        k = int(min(max((m - keys.size) * rate * 1.25, 4096), 4 * m - drawn))
        u = np.searchsorted(cdf, rng.random(k), side="right").clip(0, n - 1)
        v = np.searchsorted(cdf, rng.random(k), side="right").clip(0, n - 1)
        drawn += k
        keep = u != v
        lo = np.minimum(u[keep], v[keep]).astype(np.int64)
        hi = np.maximum(u[keep], v[keep]).astype(np.int64)
        keys = _sorted_unique(np.concatenate([keys, (lo << 32) | hi]))
    if keys.size > m:
        keys = rng.permutation(keys)[:m]
    e = np.empty((keys.size, 2), dtype=np.int32)
    e[:, 0] = (keys >> 32).astype(np.int32)
    e[:, 1] = (keys & 0xFFFFFFFF).astype(np.int32)
    return _relabel(e, n, rng)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 1) -> np.ndarray:
    """R-MAT graph on 2^scale vertices from edge_factor * 2^scale samples.

    Symmetrised (canonical u<v), self-loops and duplicates dropped, ids permuted.
    Scale 20 with edge factor 16 gives ~14M undirected edges.
    """
    rng = _rng(seed)
    n = 1 << scale
    ns = edge_factor * n
    u = np.zeros(ns, dtype=np.int64)
    v = np.zeros(ns, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for _ in range(scale):
        r = rng.random(ns, dtype=np.float32)
        bu = r >= ab                       # quadrants c, d
        bv = ((r >= a) & (r < ab)) | (r >= abc)  # quadrants b, d
        u = (u << 1) | bu
        v = (v << 1) | bv
    e = _canonical_unique(u, v)
    return _relabel(e, n, rng)


def grid2d(side: int, diag_frac: float = 0.1, seed: int = 1) -> np.ndarray:
    """side x side 4-neighbour lattice plus one random diagonal for a fraction of cells."""
    rng = _rng(seed)
    idx = np.arange(side * side, dtype=np.int64).reshape(side, side)
    right = np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], 1)
    down = np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], 1)
    cells = idx[:-1, 1:-1].ravel()
    pick = cells[rng.random(cells.size) < diag_frac]
    sgn = np.where(rng.random(pick.size) < 0.5, -1, 1)
    diag = np.stack([pick, pick + side + sgn], 1)
    allp = np.concatenate([right, down, diag])
    e = _canonical_unique(allp[:, 0], allp[:, 1])
    return _relabel(e, side * side, rng)


def erdos_renyi(n: int, m: int, seed: int = 1) -> np.ndarray:
    """Uniform random graph with up to m unique edges (small test graphs)."""
    rng = _rng(seed)
    if n < 2:
        return np.zeros((0, 2), dtype=np.int32)
    u = rng.integers(0, n, size=3 * m + 8)
    v = rng.integers(0, n, size=3 * m + 8)
    e = _canonical_unique(u, v)
    if e.shape[0] > m:
        e = e[rng.permutation(e.shape[0])[:m]]
    return e


def shuffled(edges: np.ndarray, seed: int) -> np.ndarray:
    """A seeded permutation of an edge list (one per Ins / Del stream)."""
    rng = _rng(seed)
    return edges[rng.permutation(edges.shape[0])]


def batches(edges: np.ndarray, batch: int):
    """Regular intervals of a permuted edge list, as the Ins/Del protocol takes them."""
    for s in range(0, edges.shape[0], batch):
        yield np.ascontiguousarray(edges[s:s + batch])


def mix_stream(edges: np.ndarray, batch: int, nbatches: int, load: float = 0.9,
               seed: int = 3):
    """Mixed workload: returns (preload, [(ins_i, del_i)]) on a load-fraction graph.

    The preload is ``load`` of the edges; each mixed batch inserts batch/2 edges
    from the absent pool and deletes batch/2 present edges (insert then delete,
    as a mixed update is applied).
    """
    rng = _rng(seed)
    perm = edges[rng.permutation(edges.shape[0])]
    k = int(load * edges.shape[0])
    pre = np.ascontiguousarray(perm[:k])
    present_arr = np.arange(k)
    absent_arr = np.arange(k, edges.shape[0])
    out = []
    half = batch // 2
    for _ in range(nbatches):
        ia = rng.choice(absent_arr.size, size=min(half, absent_arr.size), replace=False)
        ip = rng.choice(present_arr.size, size=min(half, present_arr.size), replace=False)
        ins_idx = absent_arr[ia]
        del_idx = present_arr[ip]
        out.append((np.ascontiguousarray(perm[ins_idx]), np.ascontiguousarray(perm[del_idx])))
        # update pools: inserted become present, deleted become absent
        keep_a = np.ones(absent_arr.size, bool)
        keep_a[ia] = False
        keep_p = np.ones(present_arr.size, bool)
        keep_p[ip] = False
        present_arr = np.concatenate([present_arr[keep_p], ins_idx])
        absent_arr = np.concatenate([absent_arr[keep_a], del_idx])
    return pre, out


def noisy_batch(edges: np.ndarray, n: int, seed: int, self_loops: int = 0,
                dups: int = 0, reversed_frac: float = 0.0) -> np.ndarray:
    """A batch with injected self-loops, duplicates and reversed (v,u) copies."""
    rng = _rng(seed)
    e = edges.copy()
    if reversed_frac > 0 and e.shape[0]:
        r = rng.random(e.shape[0]) < reversed_frac
        e[r] = e[r][:, ::-1]
    parts = [e]
    if dups and e.shape[0]:
        parts.append(e[rng.integers(0, e.shape[0], size=dups)][:, ::-1])
    if self_loops:
        s = rng.integers(0, n, size=self_loops).astype(np.int32)
        parts.append(np.stack([s, s], 1))
    out = np.concatenate(parts).astype(np.int32)
    return np.ascontiguousarray(out[rng.permutation(out.shape[0])])


# ---------------------------------------------------------------------------
# Counter-based Chung-Lu draws: draw k is a pure function of (seed, k), computed in
# int64 arithmetic whose every intermediate stays below 2^63, so numpy on the host
# and torch on the device give identical edges.  Any slice of a billion-draw stream
# can then be made on either side alone (the device generates the whole stream of
# the large configuration; the host remakes its first batches for the oracle).
# ---------------------------------------------------------------------------
_P31 = 2_147_483_647  # 2^31 - 1, prime
_H31_ROUNDS = ((16_807, 1), (1_583_458_089, 7), (784_588_716, 13), (1_222_560_079, 17))


def _h31(x, seed: int):
    """Integer hash of non-negative int64 counters x (numpy array or torch tensor)
    to [0, 2^31 - 1): an affine map of (x mod p, x div p, seed) mod p, then four
    rounds of multiply-add mod p and an xor-shift."""
    lo = x % _P31
    hi = x // _P31
    y = (lo * 1_103_515_245 + (hi * 48_271) % _P31 + (int(seed) * 69_621 + 12_345) % _P31) % _P31
    for a, b in _H31_ROUNDS:
        y = (y * a + b) % _P31
        y = y ^ (y >> 15)
    return y


class ChungLuDraws:
    """The chung_lu model (same weights, scaling to mean degree 2m/n and truncation at
    sqrt(2m)) as an indexed stream of i.i.d. endpoint pairs, with vertex ids randomly
    permuted.  Draw k is (perm[u_k], perm[v_k]) with u_k, v_k drawn proportional to
    the weights from four hashes of (seed, k); pairs come as drawn (either order,
    self-loops and repeats included, as a raw update stream carries them).

    The weights are quantised to int64 (total near 2^52) and cumulated on the host;
    each endpoint is the first index whose cumulative weight exceeds a 62-bit hash
    value reduced mod the total (exact integer searchsorted on either side)."""

    def __init__(self, n: int, m: int, gamma: float, seed: int = 1):
        if n < 2 or m <= 0:
            raise ValueError("need n >= 2 and m > 0")
        self.n, self.m, self.gamma, self.seed = int(n), int(m), float(gamma), int(seed)
        w = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (gamma - 1.0))
        cap = np.sqrt(2.0 * m)
        for _ in range(8):
            w = np.minimum(w * (2.0 * m / w.sum()), cap)
        q = np.floor(w * (float(1 << 52) / w.sum())).astype(np.int64)
        del w
        self.cw = np.cumsum(q)
        self.total = int(self.cw[-1])
        i = np.arange(n, dtype=np.int64)
        self.perm = np.argsort(_h31(i, self.seed + 1) * (1 << 32) + i, kind="stable").astype(np.int32)
        self._dev = {}

    def _endpoints(self, k, xp_search, cw):
        a = _h31(4 * k, self.seed)
        b = _h31(4 * k + 1, self.seed)
        c = _h31(4 * k + 2, self.seed)
        d = _h31(4 * k + 3, self.seed)
        ru = ((a << 31) | b) % self.total
        rv = ((c << 31) | d) % self.total
        return xp_search(cw, ru), xp_search(cw, rv)

    def draws(self, start: int, count: int, chunk: int = 1 << 22) -> np.ndarray:
        """Draws start .. start+count-1 as int32[count, 2] (host, numpy)."""
        out = np.empty((count, 2), dtype=np.int32)
        for s in range(0, count, chunk):
            c = min(chunk, count - s)
            k = np.arange(start + s, start + s + c, dtype=np.int64)
            u, v = self._endpoints(k, lambda cw, r: np.searchsorted(cw, r, side="right"), self.cw)
            out[s:s + c, 0] = self.perm[u]
            out[s:s + c, 1] = self.perm[v]
        return out

    def draws_torch(self, start: int, count: int, device="cuda", chunk: int = 1 << 25):
        """The same draws as a torch int32 [count, 2] tensor computed on `device`."""
        import torch
        dev = torch.device(device)
        if dev not in self._dev:
            self._dev[dev] = (torch.from_numpy(self.cw).to(dev), torch.from_numpy(self.perm).to(dev))
        cw, perm = self._dev[dev]
        out = torch.empty((count, 2), dtype=torch.int32, device=dev)
        for s in range(0, count, chunk):
            c = min(chunk, count - s)
            k = torch.arange(start + s, start + s + c, dtype=torch.int64, device=dev)
            u, v = self._endpoints(k, lambda t, r: torch.searchsorted(t, r, right=True), cw)
            out[s:s + c, 0] = perm[u]
            out[s:s + c, 1] = perm[v]
        return out


def shuffled_device(edges, seed: int):
    """A seeded permutation of a device edge tensor."""
    import torch
    gen = torch.Generator(device=edges.device)
    gen.manual_seed(int(seed))
    return edges[torch.randperm(edges.shape[0], generator=gen, device=edges.device)]
