// Device code of the GB300 PLDS: every step of one batch update (Algorithm 1) as
// team-parallel routines.  A "team" is either the whole grid of a cooperative
// launch (one large graph) or one thread block (one small graph of a batched
// launch); the routines only use the team's thread/warp ranks and its barrier.
//
// Build note: compiled with -Xptxas -dlcm=cg, so ordinary global loads bypass L1
// and see other blocks' writes after a barrier (all state here is written during
// the kernel by some block).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "plds_types.h"

namespace pl {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kChunk = 128;  // slots per warp chunk (32 lanes x int4)

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ int ld_volatile(const int32_t *p) { return *(volatile const int32_t *)p; }

// ---------------------------------------------------------------------------
// Teams
// ---------------------------------------------------------------------------
struct GridTeam {
    Ctl *ctl;
    int64_t limit_ns;
    __device__ int tid() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ int nthreads() const { return gridDim.x * blockDim.x; }
    __device__ int wid() const { return tid() >> 5; }
    __device__ int nwarps() const { return nthreads() >> 5; }
    __device__ int bid() const { return blockIdx.x; }
    __device__ bool leader() const { return blockIdx.x == 0 && threadIdx.x == 0; }
    // Grid-wide barrier with a bounded wait: a block that waits longer than
    // limit_ns (or sees the error word set) records kErrTimeout and leaves.
    __device__ bool sync() {
        __syncthreads();
        if (threadIdx.x == 0) {
            volatile unsigned *genp = &ctl->bar_gen;
            volatile int32_t *errp = &ctl->err;
            unsigned gen = *genp;
            __threadfence();
            unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
            if (arrived == gridDim.x - 1) {
                atomicExch(&ctl->bar_count, 0u);
                __threadfence();
                atomicAdd(&ctl->bar_gen, 1u);
            } else {
                uint64_t t0 = global_ns();
                unsigned spins = 0;
                while (*genp == gen && *errp == 0) {
                    if ((++spins & 63u) == 0 && global_ns() - t0 > (uint64_t)limit_ns) {
                        atomicOr(&ctl->err, kErrTimeout);
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
        }
        __syncthreads();
        return ld_volatile(&ctl->err) == 0;
    }
};

struct BlockTeam {
    Ctl *ctl;
    __device__ int tid() const { return threadIdx.x; }
    __device__ int nthreads() const { return blockDim.x; }
    __device__ int wid() const { return threadIdx.x >> 5; }
    __device__ int nwarps() const { return blockDim.x >> 5; }
    __device__ int bid() const { return 0; }
    __device__ bool leader() const { return threadIdx.x == 0; }
    __device__ bool sync() {
        __threadfence_block();
        __syncthreads();
        bool ok = ld_volatile(&ctl->err) == 0;
        __syncthreads();
        return ok;
    }
};

// ---------------------------------------------------------------------------
// Warp helpers (all 32 lanes must call)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_sum(int x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    return x;
}

// Position in *counter for each lane with pred, -1 otherwise (one atomic per warp).
__device__ __forceinline__ int warp_append(int32_t *counter, bool pred) {
    unsigned m = __ballot_sync(kFull, pred);
    if (m == 0) return -1;
    int leader = __ffs(m) - 1;
    int base = 0;
    if (lane_id() == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    return pred ? base + __popc(m & ((1u << lane_id()) - 1u)) : -1;
}

__device__ __forceinline__ long long warp_append64(unsigned long long *counter, bool pred) {
    unsigned m = __ballot_sync(kFull, pred);
    if (m == 0) return -1;
    int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane_id() == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    return pred ? (long long)(base + __popc(m & ((1u << lane_id()) - 1u))) : -1;
}

// Exclusive warp prefix sum; *total gets the warp total.
__device__ __forceinline__ int warp_exclusive(int x, int *total) {
    int incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, incl, o);
        if (lane_id() >= o) incl += y;
    }
    *total = __shfl_sync(kFull, incl, 31);
    return incl - x;
}

// ---------------------------------------------------------------------------
// Per-vertex open-addressing tables.  A table is cap (power of two >= 4) int32
// slots at pool + off; probing walks aligned groups of 4 slots (one int4 load)
// starting at the key's home group.  A key sits in the first group, in probe
// order, that had a free slot when it was inserted, so a lookup can stop at the
// first group that holds an EMPTY slot.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t home_group(int32_t key, int32_t cap) {
    uint32_t h = (uint32_t)key * 0x9E3779B1u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    return h & (uint32_t)((cap >> 2) - 1);
}

__device__ __forceinline__ bool table_find(const int32_t *slots, int64_t off, int32_t cap, int32_t key) {
    if (cap == 0) return false;
    const int4 *t = reinterpret_cast<const int4 *>(slots + off);
    uint32_t ng = (uint32_t)cap >> 2, gi = home_group(key, cap);
    for (uint32_t it = 0; it < ng; ++it) {
        int4 q = t[gi];
        if (q.x == key || q.y == key || q.z == key || q.w == key) return true;
        if (q.x == kEmpty || q.y == kEmpty || q.z == kEmpty || q.w == kEmpty) return false;
        gi = (gi + 1) & (ng - 1);
    }
    return false;
}

// Insert a key known to be absent; returns 1 if a tombstone was reused, 0 if an
// empty slot, -1 if the table is full (cannot happen under the load bound).
__device__ __forceinline__ int table_insert(int32_t *slots, int64_t off, int32_t cap, int32_t key) {
    int32_t *t = slots + off;
    uint32_t ng = (uint32_t)cap >> 2, gi = home_group(key, cap);
    for (uint32_t it = 0; it < ng; ++it) {
        for (int s = 0; s < 4; ++s) {
            int32_t *p = t + gi * 4 + s;
            int32_t cur = *(volatile int32_t *)p;
            while (cur == kEmpty || cur == kTomb) {
                int32_t old = atomicCAS(p, cur, key);
                if (old == cur) return cur == kTomb ? 1 : 0;
                cur = old;
            }
        }
        gi = (gi + 1) & (ng - 1);
    }
    return -1;
}

// Replace a present key by a tombstone; false if the key was not found.
__device__ __forceinline__ bool table_erase(int32_t *slots, int64_t off, int32_t cap, int32_t key) {
    if (cap == 0) return false;
    int32_t *t = slots + off;
    uint32_t ng = (uint32_t)cap >> 2, gi = home_group(key, cap);
    for (uint32_t it = 0; it < ng; ++it) {
        int4 q = reinterpret_cast<const int4 *>(t)[gi];
        int s = q.x == key ? 0 : q.y == key ? 1 : q.z == key ? 2 : q.w == key ? 3 : -1;
        if (s >= 0) {
            t[gi * 4 + s] = kTomb;
            return true;
        }
        if (q.x == kEmpty || q.y == kEmpty || q.z == kEmpty || q.w == kEmpty) return false;
        gi = (gi + 1) & (ng - 1);
    }
    return false;
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// Smallest power of two >= x, at least 4 and at most 2^30 (degrees stay below n < 2^31).
__device__ __forceinline__ int32_t next_pow2(int64_t x) {
    int32_t c = 4;
    while (c < x && c < (1 << 30)) c <<= 1;
    return c;
}

__device__ __forceinline__ int32_t sid_of(const GraphCtx &g, int32_t l) { return g.stamp_base + 1 + l; }

// Record an error bit and, for the first error only, which check raised it.
__device__ __forceinline__ void report(const GraphCtx &g, int32_t bit, int32_t site, int32_t a = 0,
                                      int32_t b = 0, int32_t c = 0) {
    if (atomicCAS(&g.ctl->err_site, 0, site) == 0) {
        g.ctl->err_info[0] = a;
        g.ctl->err_info[1] = b;
        g.ctl->err_info[2] = c;
    }
    atomicOr(&g.ctl->err, bit);
}

// ---------------------------------------------------------------------------
// Block-level exclusive scan used by the candidate sort (block 0 of the team).
// ---------------------------------------------------------------------------
__device__ int block_exclusive(int x, int *sh32, int *total) {
    int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int tot;
    int ex = warp_exclusive(x, &tot);
    if (lane == 0) sh32[w] = tot;
    __syncthreads();
    if (w == 0) {
        int v = lane < nw ? sh32[lane] : 0;
        int t2;
        int e = warp_exclusive(v, &t2);
        if (lane < nw) sh32[lane] = e;
        if (lane == 0) sh32[32] = t2;
    }
    __syncthreads();
    int r = ex + sh32[w];
    *total = sh32[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Step A1: canonicalise + validate.  Drops self-loops, keys each edge as
// (min,max), keeps one copy of each key (batch hash set), flags ids outside [0,n).
// ---------------------------------------------------------------------------
template <class Team>
__device__ void step_canonicalise(Team &T, const GraphCtx &g) {
    const int2 *e = reinterpret_cast<const int2 *>(g.edges);
    unsigned long long loops = 0;
    const int64_t mask = g.hcap - 1;
    for (int64_t i0 = (int64_t)T.wid() * 32; i0 < g.B; i0 += (int64_t)T.nwarps() * 32) {
        int64_t i = i0 + lane_id();
        bool fresh = false;
        unsigned long long key = 0;
        if (i < g.B) {
            int2 uv = e[i];
            if (uv.x < 0 || uv.x >= g.n || uv.y < 0 || uv.y >= g.n) {
                atomicOr(&g.ctl->err, kErrInvalidId);
            } else if (uv.x == uv.y) {
                loops++;
            } else {
                int32_t a = min(uv.x, uv.y), b = max(uv.x, uv.y);
                key = ((unsigned long long)(uint32_t)a << 32) | (uint32_t)b;
                int64_t h = (int64_t)(mix64(key) & (uint64_t)mask);
                for (int64_t it = 0; it <= mask; ++it) {
                    unsigned long long old = atomicCAS(&g.hset[h], kEmptyKey, key);
                    if (old == kEmptyKey) { fresh = true; break; }
                    if (old == key) break;
                    h = (h + 1) & mask;
                }
            }
        }
        long long pos = warp_append64(&g.ctl->ucount, fresh);
        if (fresh) g.ukeys[pos] = key;
    }
    if (loops) atomicAdd(&g.ctl->st[kStSelfLoops], loops);
}

// Step A1 (second half): keep insertions of absent / deletions of present edges;
// collect the touched endpoints (deduplicated by stamp) and, for insertions, the
// number of incoming edges per endpoint.
template <class Team>
__device__ void step_filter(Team &T, const GraphCtx &g) {
    const int64_t U = (int64_t)g.ctl->ucount;
    const int32_t stouch = g.stamp_base;
    unsigned long long filtered = 0;
    for (int64_t i0 = (int64_t)T.wid() * 32; i0 < U; i0 += (int64_t)T.nwarps() * 32) {
        int64_t i = i0 + lane_id();
        bool keep = false;
        unsigned long long key = 0;
        int32_t u = 0, v = 0;
        if (i < U) {
            key = g.ukeys[i];
            u = (int32_t)(key >> 32);
            v = (int32_t)(key & 0xffffffffu);
            bool present = table_find(g.slots, g.off[u], g.cap[u], v);
            keep = (g.op == kOpInsert) ? !present : present;
            if (!keep) filtered++;
        }
        long long pos = warp_append64(&g.ctl->vcount, keep);
        if (keep) g.vkeys[pos] = key;
        bool tu = keep && atomicExch(&g.stamp[u], stouch) != stouch;
        int pu = warp_append(&g.ctl->tcount, tu);
        if (tu) g.touched[pu] = u;
        bool tv = keep && atomicExch(&g.stamp[v], stouch) != stouch;
        int pv = warp_append(&g.ctl->tcount, tv);
        if (tv) g.touched[pv] = v;
        if (keep && g.op == kOpInsert) {
            atomicAdd(&g.inc[u], 1);
            atomicAdd(&g.inc[v], 1);
        }
    }
    if (filtered) atomicAdd(&g.ctl->st[kStFiltered], filtered);
}

// Step A2 (insert): tables whose load would pass load_num/load_den get a new,
// larger table.  First pass: list them and total the requested slots.
template <class Team>
__device__ void step_grow_request(Team &T, const GraphCtx &g) {
    const int32_t tc = g.ctl->tcount;
    for (int i0 = T.wid() * 32; i0 < tc; i0 += T.nwarps() * 32) {
        int i = i0 + lane_id();
        bool grow = false;
        int32_t x = 0, nc = 0;
        if (i < tc) {
            x = g.touched[i];
            int64_t live = g.deg[x], tb = g.tomb[x], in = g.inc[x], c = g.cap[x];
            if ((live + tb + in) * g.load_den > c * g.load_num) {
                nc = next_pow2(2 * (live + in));
                grow = true;
            }
        }
        int pos = warp_append(&g.ctl->mcnt[0], grow);
        if (grow) {
            g.M[0][pos] = make_int4(x, nc, 0, 0);
            atomicAdd(&g.ctl->grow_total, (unsigned long long)nc);
        }
    }
}

// Second pass (after the pool check): allocate and rehash, one warp per table.
template <class Team>
__device__ void step_grow_apply(Team &T, const GraphCtx &g) {
    const int32_t gc = g.ctl->mcnt[0];
    for (int i = T.wid(); i < gc; i += T.nwarps()) {
        int4 it = g.M[0][i];
        int32_t x = it.x, nc = it.y;
        unsigned long long noff = 0;
        if (lane_id() == 0) noff = atomicAdd(g.pool_top, (unsigned long long)nc);
        noff = __shfl_sync(kFull, noff, 0);
        int4 *nt = reinterpret_cast<int4 *>(g.slots + noff);
        for (int j = lane_id(); j < (nc >> 2); j += 32) nt[j] = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
        __syncwarp();
        __threadfence_block();
        int32_t oc = g.cap[x];
        int64_t oo = g.off[x];
        const int4 *ot = reinterpret_cast<const int4 *>(g.slots + oo);
        for (int j = lane_id(); j < (oc >> 2); j += 32) {
            int4 q = ot[j];
            if (q.x >= 0) table_insert(g.slots, (int64_t)noff, nc, q.x);
            if (q.y >= 0) table_insert(g.slots, (int64_t)noff, nc, q.y);
            if (q.z >= 0) table_insert(g.slots, (int64_t)noff, nc, q.z);
            if (q.w >= 0) table_insert(g.slots, (int64_t)noff, nc, q.w);
        }
        __syncwarp();
        if (lane_id() == 0) {
            g.off[x] = (int64_t)noff;
            g.cap[x] = nc;
            g.tomb[x] = 0;
        }
    }
}

// Steps A2+A3 (insert): put both directions into the tables and update deg, up
// (other endpoint on a level >= own) and up* (other endpoint on a level >= own-1).
template <class Team>
__device__ void step_apply_insert(Team &T, const GraphCtx &g) {
    const int64_t V = (int64_t)g.ctl->vcount;
    for (int64_t i = T.tid(); i < V; i += T.nthreads()) {
        unsigned long long key = g.vkeys[i];
        int32_t u = (int32_t)(key >> 32), v = (int32_t)(key & 0xffffffffu);
        int32_t lu = g.level[u], lv = g.level[v];
        int ru = table_insert(g.slots, g.off[u], g.cap[u], v);
        int rv = table_insert(g.slots, g.off[v], g.cap[v], u);
        if (ru < 0 || rv < 0) report(g, kErrInternal, 1, ru < 0 ? u : v, g.cap[ru < 0 ? u : v], g.deg[ru < 0 ? u : v]);
        if (ru == 1) atomicSub(&g.tomb[u], 1);
        if (rv == 1) atomicSub(&g.tomb[v], 1);
        atomicAdd(&g.deg[u], 1);
        atomicAdd(&g.deg[v], 1);
        if (lv >= lu) atomicAdd(&g.up[u], 1);
        if (lv >= lu - 1) atomicAdd(&g.upstar[u], 1);
        if (lu >= lv) atomicAdd(&g.up[v], 1);
        if (lu >= lv - 1) atomicAdd(&g.upstar[v], 1);
    }
}

// Steps A2+A3 (delete): tombstone both directions, decrement the counters.
template <class Team>
__device__ void step_apply_delete(Team &T, const GraphCtx &g) {
    const int64_t V = (int64_t)g.ctl->vcount;
    for (int64_t i = T.tid(); i < V; i += T.nthreads()) {
        unsigned long long key = g.vkeys[i];
        int32_t u = (int32_t)(key >> 32), v = (int32_t)(key & 0xffffffffu);
        int32_t lu = g.level[u], lv = g.level[v];
        bool eu = table_erase(g.slots, g.off[u], g.cap[u], v);
        bool ev = table_erase(g.slots, g.off[v], g.cap[v], u);
        if (!eu || !ev) report(g, kErrInternal, 2);
        atomicAdd(&g.tomb[u], 1);
        atomicAdd(&g.tomb[v], 1);
        atomicSub(&g.deg[u], 1);
        atomicSub(&g.deg[v], 1);
        if (lv >= lu) atomicSub(&g.up[u], 1);
        if (lv >= lu - 1) atomicSub(&g.upstar[u], 1);
        if (lu >= lv) atomicSub(&g.up[v], 1);
        if (lu >= lv - 1) atomicSub(&g.upstar[v], 1);
    }
}

// After deletions: rebuild, in place and smaller, tables that became sparse or
// full of tombstones (speed only; skipped when the scratch arena is full).
template <class Team>
__device__ void step_shrink(Team &T, const GraphCtx &g) {
    const int32_t tc = g.ctl->tcount;
    for (int i0 = T.wid() * 32; i0 < tc; i0 += T.nwarps() * 32) {
        int i = i0 + lane_id();
        int32_t x = 0, nc = 0, d = 0, c = 0;
        bool want = false;
        if (i < tc) {
            x = g.touched[i];
            d = g.deg[x];
            c = g.cap[x];
            int32_t tb = g.tomb[x];
            if (c > 4 && ((int64_t)d * 8 < c || (int64_t)tb * 4 > c)) {
                // rebuilt in place, so never larger than the current region (d < c always)
                nc = min(next_pow2(2 * (int64_t)d), c);
                want = nc < c || tb > 0;
            }
        }
        int base = -1;
        if (want) {
            base = atomicAdd(&g.ctl->shrink_used, d);
            if ((int64_t)base + d > g.arena_cap) want = false;
        }
        unsigned m = __ballot_sync(kFull, want);
        while (m) {
            int src = __ffs(m) - 1;
            m &= m - 1;
            int32_t sx = __shfl_sync(kFull, x, src), snc = __shfl_sync(kFull, nc, src);
            int32_t sc = __shfl_sync(kFull, c, src), sbase = __shfl_sync(kFull, base, src);
            int32_t sd = __shfl_sync(kFull, d, src);
            int64_t off = g.off[sx];
            int4 *t4 = reinterpret_cast<int4 *>(g.slots + off);
            int32_t *ar = g.arena + sbase;
            int written = 0;
            for (int j0 = 0; j0 < (sc >> 2); j0 += 32) {
                int j = j0 + lane_id();
                int4 q = j < (sc >> 2) ? t4[j] : make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
                int cnt = (q.x >= 0) + (q.y >= 0) + (q.z >= 0) + (q.w >= 0);
                int tot;
                int ex = warp_exclusive(cnt, &tot);
                int p = written + ex;
                // the table holds exactly deg live keys; never write past the reservation
                if (q.x >= 0 && p < sd) ar[p++] = q.x;
                if (q.y >= 0 && p < sd) ar[p++] = q.y;
                if (q.z >= 0 && p < sd) ar[p++] = q.z;
                if (q.w >= 0 && p < sd) ar[p++] = q.w;
                written += tot;
            }
            if (written != sd) {  // counters and table disagree: report, keep the table
                if (lane_id() == 0) report(g, kErrInternal, 3);
                continue;
            }
            __syncwarp();
            for (int j = lane_id(); j < (snc >> 2); j += 32) t4[j] = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
            __syncwarp();
            __threadfence_block();
            for (int j = lane_id(); j < written; j += 32) table_insert(g.slots, off, snc, ar[j]);
            __syncwarp();
            if (lane_id() == 0) {
                g.cap[sx] = snc;
                g.tomb[sx] = 0;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Mover scans: every mover's table is read either by one thread (small tables)
// or by warps in 128-slot chunks (chunks of one large table are spread over all
// warps of the team).  The callback sees each live neighbour once.
// ---------------------------------------------------------------------------
template <class Team>
__device__ __forceinline__ void enqueue_mover(Team &T, const GraphCtx &g, int par, bool is_mover, int32_t v,
                                              int32_t aux) {
    int32_t c = is_mover ? g.cap[v] : 0;
    int mi = warp_append(&g.ctl->mcnt[par], is_mover);
    if (is_mover) g.M[par][mi] = make_int4(v, aux, c, 0);
    bool small = is_mover && c <= g.thread_max_cap;
    int ti = warp_append(&g.ctl->tlcnt[par], small);
    if (small) g.TL[par][ti] = mi;
    int nch = (is_mover && !small) ? (c + kChunk - 1) / kChunk : 0;
    int tot;
    int ex = warp_exclusive(nch, &tot);
    int base = 0;
    if (tot) {
        if (lane_id() == 0) base = atomicAdd(&g.ctl->clcnt[par], tot);
        base = __shfl_sync(kFull, base, 0);
        if ((int64_t)base + tot > g.clcap) {
            if (lane_id() == 0) report(g, kErrListOverflow, 4, base, tot, (int32_t)g.clcap);
        } else {
            for (int k = 0; k < nch; ++k) g.CL[par][base + ex + k] = make_int2(mi, k);
        }
    }
}

// ---------------------------------------------------------------------------
// Step A4: insertion rounds (Algorithm 2).
// ---------------------------------------------------------------------------

// Sort the touched vertices by level (counting sort) into S; levlist gets the
// distinct levels in increasing order.  Also resets the per-batch inc counters.
template <class Team>
__device__ bool ins_sort_candidates(Team &T, const GraphCtx &g, int *sh) {
    const int32_t tc = g.ctl->tcount;
    for (int i = T.tid(); i < tc; i += T.nthreads()) {
        int32_t x = g.touched[i];
        g.inc[x] = 0;
        atomicAdd(&g.bins[g.level[x]], 1);
    }
    if (T.leader()) {
        g.ctl->mcnt[0] = 0;
        g.ctl->slevel[0] = -1;
        g.ctl->spos[0] = 0;
    }
    if (!T.sync()) return false;
    if (T.bid() == 0) {
        int run = 0, runl = 0;
        for (int b0 = 0; b0 < g.K; b0 += blockDim.x) {
            int l = b0 + threadIdx.x;
            int c = l < g.K ? g.bins[l] : 0;
            int tot, totl;
            int ex = block_exclusive(c, sh, &tot);
            int exl = block_exclusive(c > 0 ? 1 : 0, sh, &totl);
            if (l < g.K) {
                g.bins[l] = run + ex;
                if (c > 0) g.levlist[runl + exl] = l;
            }
            run += tot;
            runl += totl;
        }
        if (threadIdx.x == 0) g.ctl->nlev = runl;
    }
    if (!T.sync()) return false;
    for (int i = T.tid(); i < tc; i += T.nthreads()) {
        int32_t x = g.touched[i];
        int pos = atomicAdd(&g.bins[g.level[x]], 1);
        g.S[pos] = x;
    }
    // after the scatter bins[l] is the end of level l's range (= start of l+1)
    return T.sync();
}

// Neighbour effects of one mover v (moved from l to l+1) on one neighbour w.
struct InsNbr {
    int32_t l, snext, par;
    __device__ __forceinline__ void operator()(const GraphCtx &g, int32_t w, int &cnt_l, bool &push) const {
        int32_t raw = g.level[w];
        if (raw & kMoveFlag) return;  // w moved up in this round as well
        if (raw == l) {
            cnt_l++;
        } else if (raw == l + 1) {
            atomicAdd(&g.up[w], 1);  // v joins Z_{l+1}
            push = atomicExch(&g.stamp[w], snext) != snext;
        } else if (raw == l + 2) {
            atomicAdd(&g.upstar[w], 1);  // v joins Z_{l+1} = Z_{level(w)-1}
        }
    }
};

template <class Team>
__device__ bool ins_rounds(Team &T, const GraphCtx &g, const int32_t *sh_upmax) {
    unsigned long long visits = 0, scanned = 0;
    for (int r = 0;; ++r) {
        const int p = r & 1, q = p ^ 1;
        // which level does this round process?  (same decision in every thread)
        const int32_t fc = g.ctl->fcnt[p], sp = g.ctl->spos[p], prev = g.ctl->slevel[p];
        const int32_t sl = sp < g.ctl->nlev ? g.levlist[sp] : kInf;
        int32_t l = fc > 0 ? prev + 1 : kInf;
        if (sl < l) l = sl;
        if (l == kInf) break;
        if (l >= g.K - 1 || r > g.K + 2) {  // the top group is never violated
            if (T.leader()) report(g, kErrInternal, 5, l, r, fc);
            return false;
        }
        int32_t s_lo = 0, s_hi = 0;
        if (sl == l) {
            s_lo = l == 0 ? 0 : g.bins[l - 1];
            s_hi = g.bins[l];
        }
        if (T.leader()) {
            g.ctl->slevel[q] = l;
            g.ctl->spos[q] = sl == l ? sp + 1 : sp;
            g.ctl->mcnt[q] = 0;
            g.ctl->tlcnt[q] = 0;
            g.ctl->clcnt[q] = 0;
        }
        const int32_t scur = sid_of(g, l), snext = sid_of(g, l + 1);
        const int32_t cut = sh_upmax[l / g.Lg];
        // Phase A: candidates on level l = frontier F[p] plus initial candidates at l.
        const int32_t nitems = fc + (s_hi - s_lo);
        for (int i0 = T.wid() * 32; i0 < nitems; i0 += T.nwarps() * 32) {
            int i = i0 + lane_id();
            bool valid = i < nitems, mover = false;
            int32_t v = 0, upv = 0;
            if (valid) {
                if (i < fc) {
                    v = g.F[p][i];
                } else {
                    // skip if v is also in F: F entries carry scur, or snext once their
                    // copy has already moved v in this phase
                    v = g.S[s_lo + (i - fc)];
                    const int32_t old = atomicExch(&g.stamp[v], scur);
                    valid = old != scur && old != snext;
                }
            }
            if (valid) {
                int32_t raw = g.level[v];
                if ((raw & kLevelMask) != l) {
                    report(g, kErrInternal, 6, v, raw, l);
                } else {
                    upv = g.up[v];
                    mover = upv > cut;  // Invariant 1 violated on level l
                    if (mover) {
                        g.level[v] = (l + 1) | kMoveFlag;
                        g.upstar[v] = upv;  // Z_l is unchanged by the round: new up* = old up
                        g.stamp[v] = snext;
                    } else if (raw & kMoveFlag) {
                        g.level[v] = l;
                    }
                }
            }
            int fi = warp_append(&g.ctl->fcnt[q], mover);
            if (mover) g.F[q][fi] = v;
            enqueue_mover(T, g, p, mover, v, upv);
        }
        if (!T.sync()) return false;
        // Phase B: scan the movers' neighbours.
        if (T.leader()) {
            int32_t mc = g.ctl->mcnt[p];
            if (mc > 0) g.ctl->st[kStRounds] += 1;
            g.ctl->st[kStMoves] += (unsigned long long)mc;
            g.ctl->fcnt[p] = 0;
        }
        const InsNbr fn{l, snext, p};
        // thread-mode movers
        const int32_t tlc = g.ctl->tlcnt[p];
        for (int i0 = T.wid() * 32; i0 < tlc; i0 += T.nwarps() * 32) {
            int i = i0 + lane_id();
            int4 m = make_int4(0, 0, 0, 0);
            if (i < tlc) m = g.M[p][g.TL[p][i]];
            const int4 *t4 = reinterpret_cast<const int4 *>(g.slots + (i < tlc ? g.off[m.x] : 0));
            int ng = m.z >> 2;
            int cnt_l = 0;
            int maxg = __reduce_max_sync(kFull, (unsigned)ng);
            for (int j = 0; j < maxg; ++j) {
                int4 s4 = j < ng ? t4[j] : make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
                scanned += (j < ng) ? 4 : 0;
                int32_t ws[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    bool push = false;
                    if (ws[k] >= 0) {
                        visits++;
                        fn(g, ws[k], cnt_l, push);
                    }
                    int fi = warp_append(&g.ctl->fcnt[q], push);
                    if (push) g.F[q][fi] = ws[k];
                }
            }
            if (i < tlc && cnt_l) atomicSub(&g.up[m.x], cnt_l);
        }
        // warp chunks
        const int32_t clc = g.ctl->clcnt[p];
        for (int c = T.wid(); c < clc; c += T.nwarps()) {
            int2 it = g.CL[p][c];
            int4 m = g.M[p][it.x];
            int j = it.y * (kChunk / 4) + lane_id();
            bool in = j < (m.z >> 2);
            int4 s4 = in ? reinterpret_cast<const int4 *>(g.slots + g.off[m.x])[j]
                         : make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
            scanned += in ? 4 : 0;
            int cnt_l = 0;
            int32_t ws[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                bool push = false;
                if (ws[k] >= 0) {
                    visits++;
                    fn(g, ws[k], cnt_l, push);
                }
                int fi = warp_append(&g.ctl->fcnt[q], push);
                if (push) g.F[q][fi] = ws[k];
            }
            cnt_l = warp_sum(cnt_l);
            if (lane_id() == 0 && cnt_l) atomicSub(&g.up[m.x], cnt_l);
        }
        if (!T.sync()) return false;
    }
    visits = warp_sum64(visits);
    scanned = warp_sum64(scanned);
    if (lane_id() == 0) {
        atomicAdd(&g.ctl->st[kStVisits], visits);
        atomicAdd(&g.ctl->st[kStSlotsScanned], scanned);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Steps A5/A6: desire-level and deletion rounds (Algorithms 3 and 4).
// ---------------------------------------------------------------------------

// Desire-level of w (on level lw, violating Invariant 2), computed by one warp:
// the largest x <= lw-2 with cnt(x) >= dnmin[gn(x)], plus one, where cnt(x) is
// the number of neighbours on levels >= x; 0 if there is none.  The predicate is
// monotone in x (cnt falls, dnmin[gn(x)] rises), so the group holding the answer
// is found from per-group counts (pass 1) and the level inside it from a
// per-level histogram of that group (pass 2, 256-level windows).
__device__ int32_t warp_desire_level(const GraphCtx &g, int32_t w, int32_t lw, const int32_t *sh_dnmin,
                                     int32_t *hist) {
    if (lw < 2) return 0;
    const int32_t Lg = g.Lg, G = g.G;
    const int32_t c = g.cap[w];
    const int4 *t4 = reinterpret_cast<const int4 *>(g.slots + g.off[w]);
    const int32_t xmax = lw - 2;
    const int32_t gmax = xmax / Lg;  // groups 0..gmax start at or below xmax
    for (int k = lane_id(); k < G; k += 32) hist[k] = 0;
    __syncwarp();
    for (int j = lane_id(); j < (c >> 2); j += 32) {
        int4 q = t4[j];
        if (q.x >= 0) atomicAdd(&hist[g.level[q.x] / Lg], 1);
        if (q.y >= 0) atomicAdd(&hist[g.level[q.y] / Lg], 1);
        if (q.z >= 0) atomicAdd(&hist[g.level[q.z] / Lg], 1);
        if (q.w >= 0) atomicAdd(&hist[g.level[q.w] / Lg], 1);
    }
    __syncwarp();
    // suffix sums: cntg[i] = neighbours on levels >= i*Lg (sequential, G <= 512)
    if (lane_id() == 0) {
        int run = 0;
        for (int k = G - 1; k >= 0; --k) {
            run += hist[k];
            hist[k] = run;
        }
    }
    __syncwarp();
    int best = -1;
    for (int k0 = 0; k0 <= gmax; k0 += 32) {
        int k = k0 + lane_id();
        bool ok = k <= gmax && hist[k] >= sh_dnmin[k];
        unsigned m = __ballot_sync(kFull, ok);
        if (m) best = k0 + 31 - __clz(m);
    }
    if (best < 0) return 0;
    const int32_t need = sh_dnmin[best];
    const int32_t a = best * Lg;
    int32_t hi = min((best + 1) * Lg - 1, xmax);
    __syncwarp();
    for (;;) {
        const int32_t lo = max(a, hi - (kWindow - 1));
        for (int k = lane_id(); k < kWindow + 1; k += 32) hist[k] = 0;
        __syncwarp();
        for (int j = lane_id(); j < (c >> 2); j += 32) {
            int4 q = t4[j];
            int32_t ws[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                if (ws[s] < 0) continue;
                int32_t lu = g.level[ws[s]];
                if (lu > hi) atomicAdd(&hist[kWindow], 1);
                else if (lu >= lo) atomicAdd(&hist[lu - lo], 1);
            }
        }
        __syncwarp();
        int found = -1;
        if (lane_id() == 0) {
            int run = hist[kWindow];
            for (int x = hi; x >= lo; --x) {
                run += hist[x - lo];
                if (run >= need) { found = x; break; }
            }
        }
        found = __shfl_sync(kFull, found, 0);
        if (found >= 0) return found + 1;
        if (lo == a) return a + 1;  // unreachable: cnt(a) >= need holds
        hi = lo - 1;
        __syncwarp();
    }
}

// Initial desire-levels: touched vertices that violate Invariant 2 (level > 0 and
// up* < dnmin[gn(level-1)]) become pending.
template <class Team>
__device__ void del_initial(Team &T, const GraphCtx &g, const int32_t *sh_dnmin, int32_t *whist) {
    const int32_t tc = g.ctl->tcount;
    unsigned long long evals = 0, evisits = 0;
    for (int i0 = T.wid() * 32; i0 < tc; i0 += T.nwarps() * 32) {
        int i = i0 + lane_id();
        int32_t x = 0, lx = 0;
        bool viol = false;
        if (i < tc) {
            x = g.touched[i];
            lx = g.level[x];
            viol = lx > 0 && g.upstar[x] < sh_dnmin[(lx - 1) / g.Lg];
        }
        unsigned m = __ballot_sync(kFull, viol);
        while (m) {
            int src = __ffs(m) - 1;
            m &= m - 1;
            int32_t sx = __shfl_sync(kFull, x, src), slx = __shfl_sync(kFull, lx, src);
            int32_t d = warp_desire_level(g, sx, slx, sh_dnmin, whist);
            if (lane_id() == 0) {
                evals++;
                evisits += g.deg[sx];
                g.dlv[sx] = d;
                int pos = atomicAdd(&g.ctl->pcnt[0], 1);
                g.P[0][pos] = make_int4(sx, d, 0, 0);
                atomicMin(&g.ctl->nextmin[0], d);
            }
        }
    }
    if (evals) {
        atomicAdd(&g.ctl->st[kStDlEvals], evals);
        atomicAdd(&g.ctl->st[kStDlVisits], evisits);
    }
}

// Neighbour effects of one mover v (moved from pv down to l) on neighbour w,
// plus v's own recount (cu: neighbours >= l, cs: neighbours >= l-1).
__device__ __forceinline__ void del_nbr(const GraphCtx &g, int32_t w, int32_t l, int32_t pv, int32_t sid, int &cu,
                                        int &cs, bool &push) {
    int32_t lw = g.level[w];
    cu += lw >= l;
    cs += lw >= l - 1;
    if (lw > l) {  // w did not move this round
        if (lw <= pv) atomicSub(&g.up[w], 1);                  // v left Z_{level(w)}
        if (lw - 1 > l && lw - 1 <= pv) atomicSub(&g.upstar[w], 1);  // v left Z_{level(w)-1}
        if (lw >= l + 2 && (lw - 1 <= pv || g.dlv[w] >= 0)) push = atomicExch(&g.stamp[w], sid) != sid;
    }
}

template <class Team>
__device__ bool del_rounds(Team &T, const GraphCtx &g, const int32_t *sh_dnmin, int32_t *whist) {
    unsigned long long visits = 0, scanned = 0, evals = 0, evisits = 0;
    for (int r = 0;; ++r) {
        const int p = r & 1, q = p ^ 1;
        const int32_t l = g.ctl->nextmin[p];
        if (l == kInf) break;
        if (r > g.K + 2) {
            if (T.leader()) report(g, kErrInternal, 7);
            return false;
        }
        const int32_t sid = sid_of(g, l);
        if (T.leader()) g.ctl->rcnt[0] = 0;
        // Phase 1: pending entries with dl == l move; the rest stay pending.
        const int32_t pc = g.ctl->pcnt[p];
        for (int i0 = T.wid() * 32; i0 < pc; i0 += T.nwarps() * 32) {
            int i = i0 + lane_id();
            bool mover = false, keep = false;
            int32_t v = 0, d = 0, pv = 0;
            if (i < pc) {
                int4 e = g.P[p][i];
                v = e.x;
                d = e.y;
                if (g.dlv[v] == d) {
                    if (d == l) {
                        mover = true;
                        pv = g.level[v];
                        g.level[v] = l;
                        g.dlv[v] = -1;
                        g.up[v] = 0;
                        g.upstar[v] = 0;
                    } else {
                        keep = true;
                    }
                }
            }
            int pos = warp_append(&g.ctl->pcnt[q], keep);
            if (keep) {
                g.P[q][pos] = make_int4(v, d, 0, 0);
                atomicMin(&g.ctl->nextmin[q], d);
            }
            enqueue_mover(T, g, 0, mover, v, pv);
        }
        if (!T.sync()) return false;
        // Phase 2: movers' neighbours.
        if (T.leader()) {
            int32_t mc = g.ctl->mcnt[0];
            if (mc > 0) g.ctl->st[kStRounds] += 1;
            g.ctl->st[kStMoves] += (unsigned long long)mc;
            g.ctl->pcnt[p] = 0;
            g.ctl->nextmin[p] = kInf;
        }
        const int32_t tlc = g.ctl->tlcnt[0];
        for (int i0 = T.wid() * 32; i0 < tlc; i0 += T.nwarps() * 32) {
            int i = i0 + lane_id();
            int4 m = make_int4(0, 0, 0, 0);
            if (i < tlc) m = g.M[0][g.TL[0][i]];
            const int4 *t4 = reinterpret_cast<const int4 *>(g.slots + (i < tlc ? g.off[m.x] : 0));
            int ng = m.z >> 2;
            int cu = 0, cs = 0;
            int maxg = __reduce_max_sync(kFull, (unsigned)ng);
            for (int j = 0; j < maxg; ++j) {
                int4 s4 = j < ng ? t4[j] : make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
                scanned += (j < ng) ? 4 : 0;
                int32_t ws[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    bool push = false;
                    if (ws[k] >= 0) {
                        visits++;
                        del_nbr(g, ws[k], l, m.y, sid, cu, cs, push);
                    }
                    int ri = warp_append(&g.ctl->rcnt[0], push);
                    if (push) g.R[0][ri] = ws[k];
                }
            }
            if (i < tlc) {
                if (cu) atomicAdd(&g.up[m.x], cu);
                if (cs) atomicAdd(&g.upstar[m.x], cs);
            }
        }
        const int32_t clc = g.ctl->clcnt[0];
        for (int c = T.wid(); c < clc; c += T.nwarps()) {
            int2 it = g.CL[0][c];
            int4 m = g.M[0][it.x];
            int j = it.y * (kChunk / 4) + lane_id();
            bool in = j < (m.z >> 2);
            int4 s4 = in ? reinterpret_cast<const int4 *>(g.slots + g.off[m.x])[j]
                         : make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
            scanned += in ? 4 : 0;
            int cu = 0, cs = 0;
            int32_t ws[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                bool push = false;
                if (ws[k] >= 0) {
                    visits++;
                    del_nbr(g, ws[k], l, m.y, sid, cu, cs, push);
                }
                int ri = warp_append(&g.ctl->rcnt[0], push);
                if (push) g.R[0][ri] = ws[k];
            }
            cu = warp_sum(cu);
            cs = warp_sum(cs);
            if (lane_id() == 0) {
                if (cu) atomicAdd(&g.up[m.x], cu);
                if (cs) atomicAdd(&g.upstar[m.x], cs);
            }
        }
        if (!T.sync()) return false;
        // Phase 3: neighbours that now violate Invariant 2 get their desire-level
        // recomputed (it always lands above l).
        if (T.leader()) {
            g.ctl->mcnt[0] = 0;
            g.ctl->tlcnt[0] = 0;
            g.ctl->clcnt[0] = 0;
        }
        const int32_t rc = g.ctl->rcnt[0];
        for (int i0 = T.wid() * 32; i0 < rc; i0 += T.nwarps() * 32) {
            int i = i0 + lane_id();
            int32_t w = 0, lw = 0;
            bool viol = false;
            if (i < rc) {
                w = g.R[0][i];
                lw = g.level[w];
                viol = g.upstar[w] < sh_dnmin[(lw - 1) / g.Lg];
            }
            unsigned m = __ballot_sync(kFull, viol);
            while (m) {
                int src = __ffs(m) - 1;
                m &= m - 1;
                int32_t sw = __shfl_sync(kFull, w, src), slw = __shfl_sync(kFull, lw, src);
                int32_t d = warp_desire_level(g, sw, slw, sh_dnmin, whist);
                if (lane_id() == 0) {
                    evals++;
                    evisits += g.deg[sw];
                    if (d <= l) {
                        report(g, kErrInternal, 8);
                    } else if (d != g.dlv[sw]) {
                        g.dlv[sw] = d;
                        int pos = atomicAdd(&g.ctl->pcnt[q], 1);
                        g.P[q][pos] = make_int4(sw, d, 0, 0);
                        atomicMin(&g.ctl->nextmin[q], d);
                    }
                }
            }
        }
        if (!T.sync()) return false;
    }
    visits = warp_sum64(visits);
    scanned = warp_sum64(scanned);
    if (lane_id() == 0) {
        atomicAdd(&g.ctl->st[kStVisits], visits);
        atomicAdd(&g.ctl->st[kStSlotsScanned], scanned);
    }
    if (evals) {
        atomicAdd(&g.ctl->st[kStDlEvals], evals);
        atomicAdd(&g.ctl->st[kStDlVisits], evisits);
    }
    return true;
}

// ---------------------------------------------------------------------------
// One whole batch (Algorithm 1, one half): returns false when the team stopped
// early (error word set).  sh: shared memory with the group tables, a block-scan
// scratch and one histogram per warp.
// ---------------------------------------------------------------------------
template <class Team>
__device__ void run_batch(Team &T, const GraphCtx &g, int32_t *sh) {
    int32_t *sh_upmax = sh;
    int32_t *sh_dnmin = sh + kMaxGroups;
    int *sh_scan = sh + 2 * kMaxGroups;                     // 33 ints
    int32_t *whist = sh + 2 * kMaxGroups + 64 + (threadIdx.x >> 5) * kWarpHist;
    for (int i = threadIdx.x; i < g.G; i += blockDim.x) {
        sh_upmax[i] = g.upmax[i];
        sh_dnmin[i] = g.dnmin[i];
    }
    if (g.test_delay_us > 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        const uint64_t t0 = global_ns();  // bounded: ends after test_delay_us
        while (global_ns() - t0 < (uint64_t)g.test_delay_us * 1000u) __nanosleep(1000);
    }
    __syncthreads();
    if (g.B > 0) {
        step_canonicalise(T, g);
        if (!T.sync()) return;  // ids outside [0,n): nothing has changed
        step_filter(T, g);
        if (!T.sync()) return;
    }
    if (g.op == kOpInsert) {
        step_grow_request(T, g);
        if (!T.sync()) return;
        if (T.leader() && *g.pool_top + g.ctl->grow_total > (unsigned long long)g.pool_cap)
            atomicOr(&g.ctl->err, kErrNeedPool);  // host grows the pool and runs the batch again
        if (!T.sync()) {
            // nothing but the batch's incoming counts has changed: undo them for the rerun
            if (ld_volatile(&g.ctl->err) == kErrNeedPool)
                for (int i = T.tid(); i < g.ctl->tcount; i += T.nthreads()) g.inc[g.touched[i]] = 0;
            return;
        }
        step_grow_apply(T, g);
        if (!T.sync()) return;
        step_apply_insert(T, g);
        if (!T.sync()) return;
        if (!ins_sort_candidates(T, g, sh_scan)) return;
        ins_rounds(T, g, sh_upmax);
    } else {
        if (T.leader()) {
            g.ctl->nextmin[0] = kInf;
            g.ctl->nextmin[1] = kInf;
        }
        step_apply_delete(T, g);
        if (!T.sync()) return;
        step_shrink(T, g);
        if (!T.sync()) return;
        del_initial(T, g, sh_dnmin, whist);
        if (!T.sync()) return;
        del_rounds(T, g, sh_dnmin, whist);
    }
}

}  // namespace pl
