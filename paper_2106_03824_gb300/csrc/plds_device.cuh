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
    static constexpr bool kGrid = true;  // barriers cost a round trip to L2: fetch at the barrier
    Ctl *ctl;
    int64_t limit_ns;
    int32_t sleep_ns;
    __device__ int tid() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ int nthreads() const { return gridDim.x * blockDim.x; }
    __device__ int wid() const { return tid() >> 5; }
    __device__ int nwarps() const { return nthreads() >> 5; }
    __device__ int bid() const { return blockIdx.x; }
    __device__ int nblocks() const { return gridDim.x; }
    // a warp's rank in work lists: consecutive ranks on different blocks (SMs), so
    // that a short list spreads over the whole GPU instead of filling a few SMs
    __device__ int srank() const { return (int)(threadIdx.x >> 5) * (int)gridDim.x + (int)blockIdx.x; }
    __device__ bool leader() const { return blockIdx.x == 0 && threadIdx.x == 0; }
    // Grid-wide barrier with a bounded wait: a block that waits longer than
    // limit_ns (or sees the error word set) records kErrTimeout and leaves.
    // One 64-bit arrival counter, never reset: the k-th barrier is passed once
    // the counter reaches (k+1) x blocks.  Thread 0 of each block arrives with a
    // release add and polls with acquire loads; the block barriers around it
    // carry the other threads' writes and reads.
    __device__ bool sync() {
        __syncthreads();
        if (threadIdx.x == 0) arrive_wait();
        __syncthreads();
        return ld_volatile(&ctl->err) == 0;
    }
    // The same barrier, after which warp 0 runs fetch(lane) -- the loads the next
    // phase starts with, written to shared memory -- while lane 0 reads the error
    // word into *ok_slot: one round of loads for the block instead of a read of
    // the error word by every thread followed by the phase's own first loads.
    template <class F>
    __device__ __forceinline__ bool sync_fetch(F fetch, int32_t *ok_slot) {
        __syncthreads();
        if (threadIdx.x < 32) {
            if (threadIdx.x == 0) arrive_wait();
            __syncwarp();  // orders warp 0's loads after the acquire
            if (threadIdx.x == 0) *ok_slot = ld_volatile(&ctl->err);
            fetch((int)threadIdx.x);
        }
        __syncthreads();
        return *ok_slot == 0;
    }
    __device__ void arrive_wait() {
        {
            unsigned long long *cnt = &ctl->bar_arrivals;
            unsigned long long a;
            asm volatile("atom.add.release.gpu.global.u64 %0, [%1], 1;" : "=l"(a) : "l"(cnt) : "memory");
            const unsigned long long target = (a / gridDim.x + 1) * (unsigned long long)gridDim.x;
            volatile int32_t *errp = &ctl->err;
            uint64_t t0 = 0;
            unsigned spins = 0;
            for (;;) {
                unsigned long long v;
                asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(cnt) : "memory");
                if (v >= target || *errp != 0) break;
                if ((++spins & 63u) == 0) {
                    const uint64_t now = global_ns();
                    if (t0 == 0) {
                        t0 = now;
                    } else if (now - t0 > (uint64_t)limit_ns) {
                        atomicOr(&ctl->err, kErrTimeout);
                        break;
                    }
                }
                if (sleep_ns) __nanosleep(sleep_ns);
            }
        }
    }
};

struct BlockTeam {
    static constexpr bool kGrid = false;
    Ctl *ctl;
    __device__ int tid() const { return threadIdx.x; }
    __device__ int nthreads() const { return blockDim.x; }
    __device__ int wid() const { return threadIdx.x >> 5; }
    __device__ int nwarps() const { return blockDim.x >> 5; }
    __device__ int bid() const { return 0; }
    __device__ int nblocks() const { return 1; }
    __device__ int srank() const { return threadIdx.x >> 5; }
    __device__ bool leader() const { return threadIdx.x == 0; }
    __device__ bool sync() {
        __threadfence_block();
        __syncthreads();
        bool ok = ld_volatile(&ctl->err) == 0;
        __syncthreads();
        return ok;
    }
};

// A plain (non-cooperative) grid running one step that needs no team barrier:
// the kernel boundary orders it against the next step.
struct FreeTeam {
    static constexpr bool kGrid = false;
    __device__ int tid() const { return blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ int nthreads() const { return gridDim.x * blockDim.x; }
    __device__ int wid() const { return tid() >> 5; }
    __device__ int nwarps() const { return nthreads() >> 5; }
    __device__ int bid() const { return blockIdx.x; }
    __device__ int nblocks() const { return gridDim.x; }
    __device__ int srank() const { return (int)(threadIdx.x >> 5) * (int)gridDim.x + (int)blockIdx.x; }
    __device__ bool leader() const { return blockIdx.x == 0 && threadIdx.x == 0; }
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
// empty slot, -1 if the table is full (cannot happen under the load bound).  One
// 16-byte load per probed group, then a compare-and-swap on each free slot it
// showed (other threads may be inserting into the same table).
__device__ __forceinline__ int table_insert(int32_t *slots, int64_t off, int32_t cap, int32_t key) {
    int32_t *t = slots + off;
    uint32_t ng = (uint32_t)cap >> 2, gi = home_group(key, cap);
    for (uint32_t it = 0; it < ng; ++it) {
        const int4 q = __ldcg(reinterpret_cast<const int4 *>(t) + gi);
        const int32_t qs[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            int32_t cur = qs[s];
            while (cur == kEmpty || cur == kTomb) {
                const int32_t old = atomicCAS(t + gi * 4 + s, cur, key);
                if (old == cur) return cur == kTomb ? 1 : 0;
                cur = old;
            }
        }
        gi = (gi + 1) & (ng - 1);
    }
    return -1;
}

// Insert into a table being rebuilt (no tombstones: every slot is EMPTY or a key):
// compare-and-swap straight away, from a slot of the home group picked by the key
// so that keys sharing a group rarely race for one slot.  Any free slot of the
// first group with room is as good as another for table_find.
__device__ __forceinline__ int table_insert_fresh(int32_t *slots, int64_t off, int32_t cap, int32_t key) {
    int32_t *t = slots + off;
    const uint32_t ng = (uint32_t)cap >> 2;
    uint32_t gi = home_group(key, cap);
    const int s0 = (int)(((uint32_t)key * 0x2545F491u) >> 30);
    for (uint32_t it = 0; it < ng; ++it) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (atomicCAS(t + gi * 4 + ((s0 + k) & 3), kEmpty, key) == kEmpty) return 0;
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

__device__ __forceinline__ int4 empty4() { return make_int4(kEmpty, kEmpty, kEmpty, kEmpty); }


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

__device__ __forceinline__ int32_t sid_of(int32_t stamp_base, int32_t l) { return stamp_base + 1 + l; }

// A neighbour id read from a table; anything outside [0,n) other than the empty
// and tombstone marks would be a corrupted slot, which is never dereferenced.
__device__ __forceinline__ bool valid_id(const GraphCtx &g, int32_t w) { return (uint32_t)w < (uint32_t)g.n; }

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

// A scan item must name a vertex and a table inside the pool; a corrupted item is
// reported and skipped instead of being dereferenced.
__device__ __forceinline__ bool item_ok(const GraphCtx &g, const int4 &it, int lg) {
    const bool ok = (uint32_t)it.x < (uint32_t)g.n && lg >= 2 && lg <= 30 && it.z >= 0 &&
                    4 * (int64_t)it.z + ((int64_t)1 << lg) <= g.pool_cap;
    if (!ok) report(g, kErrInternal, 10, it.x, lg, it.z);
    return ok;
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

// Rebuild x's table (c slots, d live keys) in place as nc slots, through arena
// room at base: one warp (all lanes call).
__device__ __forceinline__ void shrink_table_warp(const GraphCtx &g, int32_t sx, int32_t snc, int32_t sc,
                                                  int32_t sbase, int32_t sd) {
    int64_t off = g.off[sx];
    int4 *t4 = reinterpret_cast<int4 *>(g.slots + off);
    int32_t *ar = g.arena + sbase;
    int written = 0;
    for (int j0 = 0; j0 < (sc >> 2); j0 += 32) {
        int j = j0 + lane_id();
        int4 q = j < (sc >> 2) ? t4[j] : empty4();
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
        return;
    }
    __syncwarp();
    for (int j = lane_id(); j < (snc >> 2); j += 32) t4[j] = empty4();
    __syncwarp();
    __threadfence_block();
    for (int j = lane_id(); j < written; j += 32) table_insert_fresh(g.slots, off, snc, ar[j]);
    __syncwarp();
    if (lane_id() == 0) {
        g.cap[sx] = snc;
        g.tomb[sx] = 0;
    }
}

// ---------------------------------------------------------------------------
// Steps A1-A2 for any team: between two steps a team barrier, or, for the
// single-graph calls, a kernel boundary (each step its own full-occupancy kernel
// with a FreeTeam).  Appends to the shared lists and room taken from the pool or
// the shrink arena are reserved once per block (block_reserve) instead of once per
// warp or thread: per-warp atomics on one counter serialise in L2.  Loops over
// lists are block-strided so that every thread of a block runs the same iterations.
// ---------------------------------------------------------------------------

// Every thread of the block calls with its amount (0: none); returns the position
// of its first entry in the list whose length is *cnt (one global atomic per
// block).  sh: blockDim.x / 32 + 1 slots of shared scratch.
template <class C>
__device__ C block_reserve(C *cnt, C amount, C *sh) {
    const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    C incl = amount;
    for (int o = 1; o < 32; o <<= 1) {
        const C y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        C run = 0;
        for (int k = 0; k < nw; ++k) {
            const C t = sh[k];
            sh[k] = run;
            run += t;
        }
        sh[nw] = run ? atomicAdd(cnt, run) : (C)0;
    }
    __syncthreads();
    const C pos = sh[nw] + sh[w] + incl - amount;
    __syncthreads();  // sh is reused by the next call
    return pos;
}

// Step A1: canonicalise + validate.  Drops self-loops, keys each edge as
// (min,max), keeps one copy of each key (batch hash set), flags ids outside [0,n).
template <class Team>
__device__ void pre_canon(Team &T, const GraphCtx &g, const BatchIn &in, unsigned long long *sh) {
    const int2 *e = reinterpret_cast<const int2 *>(in.edges);
    unsigned long long loops = 0;
    const int64_t mask = g.hcap - 1, stride = (int64_t)T.nblocks() * blockDim.x;
    for (int64_t b0 = (int64_t)T.bid() * blockDim.x; b0 < in.B; b0 += stride) {
        const int64_t i = b0 + threadIdx.x;
        bool fresh = false;
        unsigned long long key = 0;
        if (i < in.B) {
            const int2 uv = e[i];
            if (uv.x < 0 || uv.x >= g.n || uv.y < 0 || uv.y >= g.n) {
                atomicOr(&g.ctl->err, kErrInvalidId);
            } else if (uv.x == uv.y) {
                loops++;
            } else {
                const int32_t a = min(uv.x, uv.y), b = max(uv.x, uv.y);
                key = ((unsigned long long)(uint32_t)a << 32) | (uint32_t)b;
                int64_t h = (int64_t)(mix64(key) & (uint64_t)mask);
                for (int64_t it = 0; it <= mask; ++it) {
                    const unsigned long long old = atomicCAS(&g.hset[h], kEmptyKey, key);
                    if (old == kEmptyKey) { fresh = true; break; }
                    if (old == key) break;
                    h = (h + 1) & mask;
                }
            }
        }
        const unsigned long long pos = block_reserve<unsigned long long>(&g.ctl->ucount, fresh ? 1ull : 0ull, sh);
        if (fresh) g.ukeys[pos] = key;
    }
    loops = warp_sum64(loops);
    if (lane_id() == 0 && loops) atomicAdd(&g.ctl->st[kStSelfLoops], loops);
}

// Step A1, second half: keep insertions of absent / deletions of present edges;
// collect the touched endpoints (deduplicated by stamp) and, for insertions, the
// number of incoming edges per endpoint.
template <class Team>
__device__ void pre_filter(Team &T, const GraphCtx &g, const BatchIn &in, unsigned long long *sh) {
    const int64_t U = (int64_t)g.ctl->ucount, stride = (int64_t)T.nblocks() * blockDim.x;
    const int32_t stouch = in.stamp_base;
    unsigned long long filtered = 0;
    for (int64_t b0 = (int64_t)T.bid() * blockDim.x; b0 < U; b0 += stride) {
        const int64_t i = b0 + threadIdx.x;
        bool keep = false;
        unsigned long long key = 0;
        int32_t u = 0, v = 0;
        if (i < U) {
            key = g.ukeys[i];
            u = (int32_t)(key >> 32);
            v = (int32_t)(key & 0xffffffffu);
            const bool present = table_find(g.slots, g.off[u], g.cap[u], v);
            keep = (in.op == kOpInsert) ? !present : present;
            if (!keep) filtered++;
        }
        const bool tu = keep && atomicExch(&g.stamp[u], stouch) != stouch;
        const bool tv = keep && atomicExch(&g.stamp[v], stouch) != stouch;
        if (keep && in.op == kOpInsert) {
            atomicAdd(&g.inc[u], 1);
            atomicAdd(&g.inc[v], 1);
        }
        const unsigned long long pos = block_reserve<unsigned long long>(&g.ctl->vcount, keep ? 1ull : 0ull, sh);
        if (keep) g.vkeys[pos] = key;
        const unsigned long long pt =
            block_reserve<unsigned long long>(&g.ctl->ttotal, (unsigned long long)(tu + tv), sh);
        if (tu) g.touched[pt] = u;
        if (tv) g.touched[pt + (tu ? 1 : 0)] = v;
    }
    filtered = warp_sum64(filtered);
    if (lane_id() == 0 && filtered) atomicAdd(&g.ctl->st[kStFiltered], filtered);
}

// Step A1 in one pass (the single-graph calls' step kernels): the thread that puts
// a key into the batch's key set first also filters it, so the unique keys are
// counted (ucount) but never listed.  An id outside [0, n) anywhere in the batch
// stops the steps after this one; the incoming counts that valid keys left behind
// are then cleared (k_undo_inc) before the call reports the error.
template <class Team>
__device__ void pre_canon_filter(Team &T, const GraphCtx &g, const BatchIn &in, unsigned long long *sh) {
    const int2 *e = reinterpret_cast<const int2 *>(in.edges);
    const int32_t stouch = in.stamp_base;
    unsigned long long loops = 0, filtered = 0;
    const int64_t mask = g.hcap - 1, stride = (int64_t)T.nblocks() * blockDim.x;
    for (int64_t b0 = (int64_t)T.bid() * blockDim.x; b0 < in.B; b0 += stride) {
        const int64_t i = b0 + threadIdx.x;
        bool fresh = false;
        unsigned long long key = 0;
        int32_t u = 0, v = 0;
        if (i < in.B) {
            const int2 uv = e[i];
            if (uv.x < 0 || uv.x >= g.n || uv.y < 0 || uv.y >= g.n) {
                atomicOr(&g.ctl->err, kErrInvalidId);
            } else if (uv.x == uv.y) {
                loops++;
            } else {
                u = min(uv.x, uv.y);
                v = max(uv.x, uv.y);
                key = ((unsigned long long)(uint32_t)u << 32) | (uint32_t)v;
                int64_t h = (int64_t)(mix64(key) & (uint64_t)mask);
                for (int64_t it = 0; it <= mask; ++it) {
                    const unsigned long long old = atomicCAS(&g.hset[h], kEmptyKey, key);
                    if (old == kEmptyKey) { fresh = true; break; }
                    if (old == key) break;
                    h = (h + 1) & mask;
                }
            }
        }
        bool keep = false;
        if (fresh) {
            const bool present = table_find(g.slots, g.off[u], g.cap[u], v);
            keep = (in.op == kOpInsert) ? !present : present;
            if (!keep) filtered++;
        }
        block_reserve<unsigned long long>(&g.ctl->ucount, fresh ? 1ull : 0ull, sh);
        const bool tu = keep && atomicExch(&g.stamp[u], stouch) != stouch;
        const bool tv = keep && atomicExch(&g.stamp[v], stouch) != stouch;
        if (keep && in.op == kOpInsert) {
            atomicAdd(&g.inc[u], 1);
            atomicAdd(&g.inc[v], 1);
        }
        const unsigned long long pos = block_reserve<unsigned long long>(&g.ctl->vcount, keep ? 1ull : 0ull, sh);
        if (keep) g.vkeys[pos] = key;
        const unsigned long long pt =
            block_reserve<unsigned long long>(&g.ctl->ttotal, (unsigned long long)(tu + tv), sh);
        if (tu) g.touched[pt] = u;
        if (tv) g.touched[pt + (tu ? 1 : 0)] = v;
    }
    loops = warp_sum64(loops);
    filtered = warp_sum64(filtered);
    if (lane_id() == 0 && loops) atomicAdd(&g.ctl->st[kStSelfLoops], loops);
    if (lane_id() == 0 && filtered) atomicAdd(&g.ctl->st[kStFiltered], filtered);
}

// Step A2 (insert): tables whose load would pass load_num/load_den must grow:
// list them (M[0] = {x, new size}) and total their sizes.  Run after pre_filter;
// tcount is taken from its touched total.
template <class Team>
__device__ void pre_grow_request(Team &T, const GraphCtx &g, unsigned long long *sh) {
    const int32_t tc = (int32_t)g.ctl->ttotal;
    const int64_t stride = (int64_t)T.nblocks() * blockDim.x;
    if (T.leader()) g.ctl->tcount = tc;
    for (int64_t b0 = (int64_t)T.bid() * blockDim.x; b0 < tc; b0 += stride) {
        const int64_t i = b0 + threadIdx.x;
        bool grow = false;
        int32_t x = 0, nc = 0;
        if (i < tc) {
            x = g.touched[i];
            const int64_t live = g.deg[x], tb = g.tomb[x], in = g.inc[x], c = g.cap[x];
            if ((live + tb + in) * g.load_den > c * g.load_num) {
                nc = next_pow2(2 * (live + in));
                grow = true;
            }
        }
        const unsigned long long pos = block_reserve<unsigned long long>(&g.ctl->gtotal, grow ? 1ull : 0ull, sh);
        if (grow) g.M[0][pos] = make_int4(x, nc, 0, 0);
        block_reserve<unsigned long long>(&g.ctl->grow_total, grow ? (unsigned long long)nc : 0ull, sh);
    }
}

// The pool check before any table moves: every thread reads the same pool top,
// since nothing is taken from the pool in this step.  When the pool cannot
// take the growing tables, the batch's incoming counts are undone and the host
// grows the pool and runs the batch again.
template <class Team>
__device__ void pre_pool_check(Team &T, const GraphCtx &g) {
    const unsigned long long top = *g.pool_top;
    if (top + g.ctl->grow_total <= (unsigned long long)g.pool_cap) {
        if (T.leader()) g.ctl->pool_old = top;  // the new tables will fill [top, top + grow_total)
        return;
    }
    for (int i = T.tid(); i < g.ctl->tcount; i += T.nthreads()) g.inc[g.touched[i]] = 0;
    if (T.leader()) atomicOr(&g.ctl->err, kErrNeedPool);
}

// Room in the pool for every growing table (after the check), and the
// work list of the move: every old table cut into chunks of kMoveChunk slots,
// items {growing-table index, chunk} in CL[0].  The rooms are contiguous from the
// pool top read by the check.
constexpr int kGrowChunk = 512;  // shrinking: slots per chunk item
constexpr int kMoveChunk = 128;  // growth: old slots per chunk item (one 16-byte group per lane)

template <class Team>
__device__ void pre_alloc(Team &T, const GraphCtx &g, unsigned long long *sh) {
    const int64_t gc = (int64_t)g.ctl->gtotal, stride = (int64_t)T.nblocks() * blockDim.x;
    for (int64_t b0 = (int64_t)T.bid() * blockDim.x; b0 < gc; b0 += stride) {
        const int64_t i = b0 + threadIdx.x;
        const int4 it = i < gc ? g.M[0][i] : make_int4(0, 0, 0, 0);
        const unsigned long long off =
            block_reserve<unsigned long long>(g.pool_top, i < gc ? (unsigned long long)it.y : 0ull, sh);
        const int32_t nch = i < gc ? (g.cap[it.x] + kMoveChunk - 1) / kMoveChunk : 0;
        const unsigned long long c0 = block_reserve<unsigned long long>(&g.ctl->ctotal, (unsigned long long)nch, sh);
        if (i < gc) {
            g.M[0][i] = make_int4(it.x, it.y, (int32_t)(off & 0xffffffffu), (int32_t)(off >> 32));
            for (int32_t k = 0; k < nch; ++k) {
                if ((int64_t)(c0 + k) < g.clcap) g.CL[0][c0 + k] = make_int4((int32_t)i, k, 0, 0);
                else report(g, kErrListOverflow, 23, (int32_t)i, k, 0);
            }
        }
    }
}

// Every new table starts empty: one fill of the contiguous rooms.
template <class Team>
__device__ void pre_clear(Team &T, const GraphCtx &g) {
    int4 *p = reinterpret_cast<int4 *>(g.slots + g.ctl->pool_old);
    const int64_t n4 = (int64_t)(g.ctl->grow_total >> 2);
    for (int64_t j = T.tid(); j < n4; j += T.nthreads()) p[j] = empty4();
}

// The old entries go into the new tables, one warp per chunk of an old table (a
// hub's table is spread over many warps).  The vertices still point at their old
// tables; pre_commit repoints them afterwards.
template <class Team>
__device__ void pre_grow(Team &T, const GraphCtx &g) {
    const int64_t nc_items = (int64_t)g.ctl->ctotal;
    for (int64_t c = T.wid(); c < nc_items; c += T.nwarps()) {
        const int4 ci = g.CL[0][c];
        const int4 it = g.M[0][ci.x];
        const int64_t noff = (int64_t)(uint32_t)it.z | ((int64_t)it.w << 32);
        const int32_t oc = g.cap[it.x];
        const int4 *ot = reinterpret_cast<const int4 *>(g.slots + g.off[it.x]);
        const int j_end = min(oc, (ci.y + 1) * kMoveChunk) >> 2;
        for (int j = (ci.y * kMoveChunk >> 2) + lane_id(); j < j_end; j += 32) {
            const int4 q = ot[j];
            if (q.x >= 0) table_insert_fresh(g.slots, noff, it.y, q.x);
            if (q.y >= 0) table_insert_fresh(g.slots, noff, it.y, q.y);
            if (q.z >= 0) table_insert_fresh(g.slots, noff, it.y, q.z);
            if (q.w >= 0) table_insert_fresh(g.slots, noff, it.y, q.w);
        }
    }
}

// Every growing vertex points at its new table.
template <class Team>
__device__ void pre_commit(Team &T, const GraphCtx &g) {
    const int64_t gc = (int64_t)g.ctl->gtotal;
    for (int64_t i = T.tid(); i < gc; i += T.nthreads()) {
        const int4 it = g.M[0][i];
        g.off[it.x] = (int64_t)(uint32_t)it.z | ((int64_t)it.w << 32);
        g.cap[it.x] = it.y;
        g.tomb[it.x] = 0;
    }
}

__device__ __forceinline__ void shrink_item(const GraphCtx &g, int list, unsigned long long pos, int32_t j, int32_t k) {
    if ((int64_t)pos < g.clcap) g.CL[list][pos] = make_int4(j, k, 0, 0);
    else report(g, kErrListOverflow, 24, j, k, list);
}

// Shrink plan (after the deletions): tables that became sparse or full of
// tombstones get arena room for their live keys and go to the warp list (M[0])
// or, above block_cap slots, the large list (M[1]) as {x, new size, arena base,
// live keys}, whose rebuild is cut into chunks; speed only, skipped when the
// arena is full.
template <class Team>
__device__ void pre_shrink_plan(Team &T, const GraphCtx &g, unsigned long long *sh) {
    const int32_t tc = (int32_t)g.ctl->ttotal;
    const int64_t stride = (int64_t)T.nblocks() * blockDim.x;
    if (T.leader()) g.ctl->tcount = tc;
    for (int64_t b0 = (int64_t)T.bid() * blockDim.x; b0 < tc; b0 += stride) {
        const int64_t i = b0 + threadIdx.x;
        int32_t x = 0, nc = 0, d = 0, c = 0;
        bool want = false;
        if (i < tc) {
            x = g.touched[i];
            d = g.deg[x];
            c = g.cap[x];
            const int32_t tb = g.tomb[x];
            if (c > 4 && ((int64_t)d * 8 < c || (int64_t)tb * 4 > c)) {
                nc = min(next_pow2(2 * (int64_t)d), c);  // in place: never larger than the region
                want = nc < c || tb > 0;
            }
        }
        const unsigned long long base =
            block_reserve<unsigned long long>(&g.ctl->atotal, want ? (unsigned long long)d : 0ull, sh);
        if (want && (int64_t)base + d > g.arena_cap) want = false;
        const bool big = want && c > g.block_cap;
        const unsigned long long ps = block_reserve<unsigned long long>(&g.ctl->gtotal, (want && !big) ? 1ull : 0ull, sh);
        const unsigned long long pb = block_reserve<unsigned long long>(&g.ctl->btotal, big ? 1ull : 0ull, sh);
        if (want && !big) g.M[0][ps] = make_int4(x, nc, (int32_t)base, d);
        if (big) {
            g.M[1][pb] = make_int4(x, nc, (int32_t)base, d);
            g.lfill[0][x] = 0;  // cursor of the compaction into the arena room
        }
        // a large table's work in chunks of kGrowChunk: compaction of its c slots,
        // clearing of its nc new slots, insertion of its d keys (lists CL[0..2])
        const int32_t n0 = big ? (c + kGrowChunk - 1) / kGrowChunk : 0;
        const int32_t n1 = big ? (nc + kGrowChunk - 1) / kGrowChunk : 0;
        const int32_t n2 = big ? (d + kGrowChunk - 1) / kGrowChunk : 0;
        const unsigned long long c0 = block_reserve<unsigned long long>(&g.ctl->ctotal, (unsigned long long)n0, sh);
        const unsigned long long c1 = block_reserve<unsigned long long>(&g.ctl->c1total, (unsigned long long)n1, sh);
        const unsigned long long c2 = block_reserve<unsigned long long>(&g.ctl->c2total, (unsigned long long)n2, sh);
        for (int32_t k = 0; k < n0; ++k) shrink_item(g, 0, c0 + k, (int32_t)pb, k);
        for (int32_t k = 0; k < n1; ++k) shrink_item(g, 1, c1 + k, (int32_t)pb, k);
        for (int32_t k = 0; k < n2; ++k) shrink_item(g, 2, c2 + k, (int32_t)pb, k);
    }
}

// Shrink, first pass: the small tables rebuilt whole, one warp each; the large
// tables' live keys copied into their arena room, one warp per chunk of slots.
template <class Team>
__device__ void pre_shrink_a(Team &T, const GraphCtx &g) {
    const int32_t sc = (int32_t)g.ctl->gtotal;
    for (int i = T.wid(); i < sc; i += T.nwarps()) {
        const int4 it = g.M[0][i];
        shrink_table_warp(g, it.x, it.y, g.cap[it.x], it.z, it.w);
    }
    const int64_t n0 = (int64_t)g.ctl->ctotal;
    for (int64_t c = T.wid(); c < n0; c += T.nwarps()) {
        const int4 ci = g.CL[0][c];
        const int4 it = g.M[1][ci.x];
        const int32_t oc = g.cap[it.x];
        const int4 *t4 = reinterpret_cast<const int4 *>(g.slots + g.off[it.x]);
        const int j = (ci.y * kGrowChunk >> 2) + lane_id();  // kGrowChunk = 4 x 32 x 4 slots
        int32_t ks[16];
        int cnt = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int4 q = (j + 32 * u) < (oc >> 2) && (j + 32 * u) < ((ci.y + 1) * kGrowChunk >> 2) ? t4[j + 32 * u]
                                                                                                     : empty4();
            ks[4 * u] = q.x; ks[4 * u + 1] = q.y; ks[4 * u + 2] = q.z; ks[4 * u + 3] = q.w;
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) cnt += ks[q] >= 0;
        int tot;
        const int ex = warp_exclusive(cnt, &tot);
        int base = 0;
        if (lane_id() == 0 && tot) base = atomicAdd(&g.lfill[0][it.x], tot);
        int p = __shfl_sync(kFull, base, 0) + ex;
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (ks[q] >= 0) {
                if (p < it.w) g.arena[it.z + p] = ks[q];  // never past the room (checked below)
                ++p;
            }
    }
}

// Shrink, second pass: a large table whose copy holds exactly its live keys is
// cleared (its first nc slots) and takes its new size; otherwise it is reported
// and kept.
template <class Team>
__device__ void pre_shrink_b(Team &T, const GraphCtx &g) {
    const int64_t n1 = (int64_t)g.ctl->c1total;
    for (int64_t c = T.wid(); c < n1; c += T.nwarps()) {
        const int4 ci = g.CL[1][c];
        const int4 it = g.M[1][ci.x];
        if (g.lfill[0][it.x] != it.w) {
            if (ci.y == 0 && lane_id() == 0) report(g, kErrInternal, 3, it.x, g.lfill[0][it.x], it.w);
            continue;
        }
        int4 *t4 = reinterpret_cast<int4 *>(g.slots + g.off[it.x]);
        const int j_end = min(it.y, (ci.y + 1) * kGrowChunk) >> 2;
        for (int j = (ci.y * kGrowChunk >> 2) + lane_id(); j < j_end; j += 32) t4[j] = empty4();
        if (ci.y == 0 && lane_id() == 0) {
            g.cap[it.x] = it.y;
            g.tomb[it.x] = 0;
        }
    }
}

// Shrink, third pass: the copied keys go back into the cleared tables, one warp
// per chunk of keys.
template <class Team>
__device__ void pre_shrink_c(Team &T, const GraphCtx &g) {
    const int64_t n2 = (int64_t)g.ctl->c2total;
    for (int64_t c = T.wid(); c < n2; c += T.nwarps()) {
        const int4 ci = g.CL[2][c];
        const int4 it = g.M[1][ci.x];
        if (g.lfill[0][it.x] != it.w) continue;  // reported and kept in the second pass
        const int64_t off = g.off[it.x];
        const int k_end = min(it.w, (ci.y + 1) * kGrowChunk);
        for (int k = ci.y * kGrowChunk + lane_id(); k < k_end; k += 32)
            table_insert_fresh(g.slots, off, it.y, g.arena[it.z + k]);
    }
}


// ---------------------------------------------------------------------------
// Mover scans.  Each moving vertex's table is scanned either by one thread
// (tables of at most thread_max_cap slots) or in 128-slot chunks, one warp per
// chunk, the chunks of a large table spread over all warps of the team.  A scan
// item is self-contained -- {vertex, table size (log2) and chunk, table offset in
// int4 units, aux} -- so a warp goes from the item straight to the slots and
// then to the neighbours' levels, with all loads of one step issued together.
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// Block-staged list appends.  Thousands of warps appending to one global list
// would serialise on its counter (same-address atomics in one L2 slice), so a
// warp claims room in its block's shared-memory buffer with a shared atomic, and
// at the end of the phase the block publishes the buffer with one global atomic
// (stage_flush).  A warp that finds the buffer full appends to the global list
// directly.  hdr[0] = staged count, hdr[1] = end of the valid staged prefix.
// ---------------------------------------------------------------------------
template <class V>
struct Stage {
    V *buf;          // shared buffer
    int32_t *hdr;    // shared {count, valid end}
    int32_t cap;     // buffer capacity
    int32_t *gcnt;   // global count
    V *glist;        // global list
    int64_t gcap;    // global capacity
};

// Reserve `cnt` consecutive entries for a warp (called by one lane); returns the
// position and whether it is in the shared buffer.
template <class V>
__device__ __forceinline__ int stage_reserve(const Stage<V> &s, int cnt, bool &shared) {
    int pos = atomicAdd(&s.hdr[0], cnt);
    if (pos + cnt <= s.cap) {
        shared = true;
        return pos;
    }
    atomicMin(&s.hdr[1], pos);  // staged entries are valid only below the first overflow
    shared = false;
    return atomicAdd(s.gcnt, cnt);
}

template <class V>
__device__ __forceinline__ void stage_put(const Stage<V> &s, bool shared, int pos, const V &x) {
    if (shared) s.buf[pos] = x;
    else if (pos < s.gcap) s.glist[pos] = x;
}

// Every lane with pred appends x (one reservation per warp).
template <class V>
__device__ __forceinline__ void stage_push(const Stage<V> &s, bool pred, const V &x) {
    const unsigned m = __ballot_sync(kFull, pred);
    if (m == 0) return;
    const int lane = lane_id(), leader = __ffs(m) - 1;
    int pos = 0;
    bool sh = false;
    if (lane == leader) pos = stage_reserve(s, __popc(m), sh);
    pos = __shfl_sync(kFull, pos, leader);
    sh = __shfl_sync(kFull, sh, leader);
    if (pred) stage_put(s, sh, pos + __popc(m & ((1u << lane) - 1u)), x);
}

// Every lane appends the entries of ws flagged in its mask.
template <int N>
__device__ __forceinline__ void stage_push_masked(const Stage<int32_t> &s, unsigned mask, const int32_t (&ws)[N]) {
    int tot;
    const int ex = warp_exclusive(__popc(mask), &tot);
    if (tot == 0) return;
    int pos = 0;
    bool sh = false;
    if (lane_id() == 0) pos = stage_reserve(s, tot, sh);
    pos = __shfl_sync(kFull, pos, 0) + ex;
    sh = __shfl_sync(kFull, sh, 0);
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (mask >> k & 1u) stage_put(s, sh, pos++, ws[k]);
}

// Publish the block's staged entries (all threads of the block call).
template <class V>
__device__ __forceinline__ void stage_flush(const GraphCtx &g, const Stage<V> &s, int32_t *tmp) {
    __syncthreads();
    const int n = min(s.hdr[0], s.hdr[1]);
    if (threadIdx.x == 0) {
        const int base = n > 0 ? atomicAdd(s.gcnt, n) : 0;
        if ((int64_t)base + n > s.gcap || (int64_t)s.gcnt[0] > s.gcap) report(g, kErrListOverflow, 4, base, n, (int32_t)s.gcap);
        *tmp = base;
    }
    __syncthreads();
    const int base = *tmp;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (base + i < s.gcap) s.glist[base + i] = s.buf[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        s.hdr[0] = 0;
        s.hdr[1] = s.cap;
    }
    __syncthreads();
}

constexpr int kStageF = 2048, kStageTL = 1024, kStageCL = 2048, kStagePK = 1024;

// Shared-memory staging of one round: frontier / recompute list, thread-mode and
// chunk scan items, pending entries, the block's mover count, and what warp 0
// fetches for the next phase while it passes the team barrier (ph4: one item per
// warp; phs: words).
struct RoundStage {
    Stage<int32_t> f;
    Stage<int4> tl, cl, pk;
    int32_t *movers;  // shared mover count of the block
    int32_t *bmin;    // shared minimum pending level of the block
    int32_t *tmp;
    int4 *ph4;
    int32_t *phs;
    int32_t *ff;             // block's climbing movers: {count, smallest new up-degree, lowest other level}
    unsigned long long *ff64;  // their {degree sum, new up-degree sum}
};

// Shared ints of a staging area whose capacities are the defaults >> shift
// (a block-sized team, alone on its graph, needs far less room than a grid).
__host__ __device__ constexpr int stage_ints(int shift) {
    return 128 + (kStageF >> shift) + 4 * ((kStageTL >> shift) + (kStageCL >> shift) + (kStagePK >> shift));
}

// Lay out the staging area (stage_ints(shift) ints of shared memory, 16-byte aligned).
__device__ __forceinline__ RoundStage stage_setup(int32_t *base, int shift) {
    RoundStage st{};
    const int cf = kStageF >> shift, ct = kStageTL >> shift, cc = kStageCL >> shift, cp = kStagePK >> shift;
    int32_t *hdr = base;
    st.ph4 = reinterpret_cast<int4 *>(base + 32);  // 16 int4
    st.phs = base + 96;                             // 32 ints
    st.f.buf = base + 128;
    st.tl.buf = reinterpret_cast<int4 *>(base + 128 + cf);
    st.cl.buf = st.tl.buf + ct;
    st.pk.buf = st.cl.buf + cc;
    st.f.hdr = hdr;
    st.tl.hdr = hdr + 2;
    st.cl.hdr = hdr + 4;
    st.pk.hdr = hdr + 6;
    st.f.cap = cf;
    st.tl.cap = ct;
    st.cl.cap = cc;
    st.pk.cap = cp;
    st.movers = hdr + 8;
    st.bmin = hdr + 9;
    st.tmp = hdr + 10;  // 4 ints
    st.ff = hdr + 14;   // 3 ints
    st.ff64 = reinterpret_cast<unsigned long long *>(hdr + 18);  // 2 x 64 bit
    if (threadIdx.x == 0) {
        hdr[0] = 0; hdr[1] = cf;
        hdr[2] = 0; hdr[3] = ct;
        hdr[4] = 0; hdr[5] = cc;
        hdr[6] = 0; hdr[7] = cp;
        hdr[8] = 0; hdr[9] = kInf;
        hdr[14] = 0; hdr[15] = kInf; hdr[16] = kInf;
        st.ff64[0] = 0;
        st.ff64[1] = 0;
    }
    __syncthreads();
    return st;
}


__device__ __forceinline__ void stage_init(int32_t *hdr, int cap) {
    hdr[0] = 0;
    hdr[1] = cap;
}

// Publish the selected lists of a phase (bit 0 f, 1 tl, 2 cl, 3 pk) together:
// warp k reserves list k's global range, then the block copies all of them.
// The headers are reset at the end; the next use comes after a team barrier.
template <class V>
__device__ __forceinline__ void stage_reserve_global(const GraphCtx &g, const Stage<V> &s, int32_t *base_out) {
    const int n = min(s.hdr[0], s.hdr[1]);
    const int base = n > 0 ? atomicAdd(s.gcnt, n) : 0;
    if ((int64_t)base + n > s.gcap) report(g, kErrListOverflow, 4, base, n, (int32_t)s.gcap);
    *base_out = base;
}

template <class V>
__device__ __forceinline__ void stage_copy_out(const Stage<V> &s, int base) {
    const int n = min(s.hdr[0], s.hdr[1]);
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (base + i < s.gcap) s.glist[base + i] = s.buf[i];
}

__device__ __forceinline__ void stage_flush_round(const GraphCtx &g, const RoundStage &st, unsigned which) {
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        const int w = threadIdx.x >> 5;
        if (w == 0 && (which & 1u)) stage_reserve_global(g, st.f, st.tmp + 0);
        if (w == 1 && (which & 2u)) stage_reserve_global(g, st.tl, st.tmp + 1);
        if (w == 2 && (which & 4u)) stage_reserve_global(g, st.cl, st.tmp + 2);
        if (w == 3 && (which & 8u)) stage_reserve_global(g, st.pk, st.tmp + 3);
    }
    __syncthreads();
    if (which & 1u) stage_copy_out(st.f, st.tmp[0]);
    if (which & 2u) stage_copy_out(st.tl, st.tmp[1]);
    if (which & 4u) stage_copy_out(st.cl, st.tmp[2]);
    if (which & 8u) stage_copy_out(st.pk, st.tmp[3]);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (which & 1u) { st.f.hdr[0] = 0; st.f.hdr[1] = st.f.cap; }
        if (which & 2u) { st.tl.hdr[0] = 0; st.tl.hdr[1] = st.tl.cap; }
        if (which & 4u) { st.cl.hdr[0] = 0; st.cl.hdr[1] = st.cl.cap; }
        if (which & 8u) { st.pk.hdr[0] = 0; st.pk.hdr[1] = st.pk.cap; }
    }
}

// Queue the scan of a mover's table; wsm: 160 ints of per-warp shared scratch.
__device__ __forceinline__ void enqueue_mover(const GraphCtx &g, const RoundStage &st, bool is_mover, int32_t v,
                                              int32_t aux, int32_t c, int64_t off, int32_t *wsm) {
    const int lane = lane_id();
    const unsigned mm = __ballot_sync(kFull, is_mover);
    if (mm == 0) return;
    if (lane == __ffs(mm) - 1) atomicAdd(st.movers, __popc(mm));
    const int lg = is_mover ? __ffs(c) - 1 : 0;
    const int32_t goff = (int32_t)(off >> 2);
    const bool small = is_mover && c <= g.thread_max_cap;
    stage_push(st.tl, small, make_int4(v, lg, goff, aux));
    const int nch = (is_mover && !small) ? (c + kChunk - 1) / kChunk : 0;
    int tot;
    const int ex = warp_exclusive(nch, &tot);
    if (tot == 0) return;
    int pos = 0;
    bool sh = false;
    if (lane == 0) pos = stage_reserve(st.cl, tot, sh);
    pos = __shfl_sync(kFull, pos, 0);
    sh = __shfl_sync(kFull, sh, 0);
    // the warp writes all its chunk items together (a large table has many)
    wsm[lane] = ex;
    wsm[32 + lane] = v;
    wsm[64 + lane] = lg;
    wsm[96 + lane] = goff;
    wsm[128 + lane] = aux;
    __syncwarp();
    for (int t = lane; t < tot; t += 32) {
        int lo = 0, hi = 31;  // owner: the last lane whose range starts at or before t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (wsm[mid] <= t) lo = mid; else hi = mid - 1;
        }
        stage_put(st.cl, sh, pos + t,
                  make_int4(wsm[32 + lo], ((t - wsm[lo]) << 5) | wsm[64 + lo], wsm[96 + lo], wsm[128 + lo]));
    }
    __syncwarp();
}

// Insertion: queue the scans of the lanes' movers of the next level.  A mover whose
// table has at most thread_max_cap slots is scanned by one thread; any other is
// scanned in 128-entry chunks, from its table (ilen < 0) or from its up-list of
// ilen entries at int4 offset ioff4 of the list buffer the round writes (a mover
// that keeps climbing), and gets room for rsize entries in list buffer k1 mod 3 for the
// neighbours that stay relevant after its move (lout = -1 when the buffer is full:
// the next scan then reads the table again).  Chunk items of a list carry 31 as
// their table size and the list length as aux.
__device__ __forceinline__ void enqueue_ins(const GraphCtx &g, const RoundStage &st, bool is_mover, int32_t v,
                                            int32_t c, int64_t off, int32_t ilen, int32_t ioff4, int32_t rsize,
                                            int k1, int32_t *wsm) {
    const int abuf = k1 % 3;  // k1: index of the phase that scans these movers
    const int lane = lane_id();
    const unsigned mm = __ballot_sync(kFull, is_mover);
    if (mm == 0) return;
    if (lane == __ffs(mm) - 1) atomicAdd(st.movers, __popc(mm));
    const bool list = is_mover && ilen >= 0;
    const bool small = is_mover && !list && c <= g.thread_max_cap;
    const int lg = (is_mover && !list) ? __ffs(c) - 1 : 31;
    const int32_t goff = list ? ioff4 : (int32_t)(off >> 2);
    stage_push(st.tl, small, make_int4(v, lg, goff, 0));
    const bool chunked = is_mover && !small;
    const bool want = chunked && (list || c >= g.list_cap);  // smaller tables: rescanning is cheaper
    int tot4;
    const int ex4 = warp_exclusive(want ? (rsize + 3) >> 2 : 0, &tot4);
    unsigned long long lbase = 0;
    if (lane == 0 && tot4 > 0) lbase = atomicAdd(&g.ctl->ltop[abuf], (unsigned long long)tot4);
    lbase = __shfl_sync(kFull, lbase, 0);
    if (chunked) {
        const bool fits = want && lbase + (unsigned long long)tot4 <= (unsigned long long)(g.lcap >> 2);
        g.lout[v] = fits ? (int32_t)(lbase + (unsigned long long)ex4) : -1;
        g.lfill[k1 & 1][v] = 0;  // the next phase's counters: last used two phases ago
    }
    const int nch = chunked ? (list ? max(1, (ilen + kChunk - 1) / kChunk) : (c + kChunk - 1) / kChunk) : 0;
    int tot;
    const int ex = warp_exclusive(nch, &tot);
    if (tot == 0) return;
    int pos = 0;
    bool sh = false;
    if (lane == 0) pos = stage_reserve(st.cl, tot, sh);
    pos = __shfl_sync(kFull, pos, 0);
    sh = __shfl_sync(kFull, sh, 0);
    wsm[lane] = ex;
    wsm[32 + lane] = v;
    wsm[64 + lane] = lg;
    wsm[96 + lane] = goff;
    wsm[128 + lane] = list ? ilen : 0;
    __syncwarp();
    for (int t = lane; t < tot; t += 32) {
        int lo = 0, hi = 31;  // owner: the last lane whose range starts at or before t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (wsm[mid] <= t) lo = mid; else hi = mid - 1;
        }
        stage_put(st.cl, sh, pos + t,
                  make_int4(wsm[32 + lo], ((t - wsm[lo]) << 5) | wsm[64 + lo], wsm[96 + lo], wsm[128 + lo]));
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Step A4: insertion rounds (Algorithm 2).
// ---------------------------------------------------------------------------

// Sort the touched vertices by level (counting sort) into S; levlist gets the
// distinct levels in increasing order.  Also resets the per-batch inc counters.
template <class Team>
__device__ bool ins_sort_candidates(Team &T, const GraphCtx &g, int *sh) {
    const int32_t tc = g.ctl->tcount;
    for (int i0 = T.wid() * 32; i0 < tc; i0 += T.nwarps() * 32) {
        const int i = i0 + lane_id();
        const int32_t x = i < tc ? g.touched[i] : 0;
        const int32_t lx = i < tc ? g.level[x] : -1;
        if (i < tc) g.inc[x] = 0;
        const unsigned peers = __match_any_sync(kFull, lx);  // lanes with the same level add once
        if (i < tc && lane_id() == __ffs(peers) - 1) atomicAdd(&g.bins[lx], __popc(peers));
    }
    if (T.leader()) g.ctl->mcnt[0] = 0;
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
    for (int i0 = T.wid() * 32; i0 < tc; i0 += T.nwarps() * 32) {
        const int i = i0 + lane_id();
        const int32_t x = i < tc ? g.touched[i] : 0;
        const int32_t lx = i < tc ? g.level[x] : -1;
        const unsigned peers = __match_any_sync(kFull, lx);
        const int leader = __ffs(peers) - 1;
        int pos = 0;
        if (i < tc && lane_id() == leader) pos = atomicAdd(&g.bins[lx], __popc(peers));
        pos = __shfl_sync(kFull, pos, leader) + __popc(peers & ((1u << lane_id()) - 1u));
        if (i < tc) g.S[pos] = x;
    }
    // after the scatter bins[l] is the end of level l's range (= start of l+1)
    return T.sync();
}

// ---------------------------------------------------------------------------
// Insertion rounds, one team barrier per level.
//
// Round l moves the movers of level l (the vertices on l that violate Invariant
// 1) to l + 1 and applies their effects: a neighbour left on l is no longer an
// up-neighbour of the mover; a neighbour on l + 1 gains an up-neighbour; one on
// l + 2 gains an up*-neighbour.  The movers of level l + 1 are found while round l
// runs, so no separate candidate phase is needed:
//   - a vertex on l + 1 that is not an initial candidate satisfies Invariant 1
//     before round l and its up-degree only grows during it, so it violates on
//     l + 1 exactly when one arrival takes its up-degree past the cutoff: the
//     thread whose atomic add sees the old value equal to the cutoff marks it;
//   - initial candidates on l + 1 are tested during round l (up-degrees only grow,
//     so a test that passes is final; one that fails is caught by the arrival
//     that crosses);
//   - a mover of level l violates again on l + 1 iff its up-degree minus its
//     neighbours left on l exceeds the cutoff; the scan of its last table chunk
//     (per-vertex chunk counter) decides, nobody else touching its up-degree.
// Movers of level l carry the flag of l's parity in their level word from their
// marking (during round l - 1, where they still read as level l) until the end of
// round l, whose readers see "mover of l" for a word with that flag and level l or
// l + 1; the flag of the other parity is ignored.  A level with no movers jumps
// to the next initial-candidate level, tested in a phase of its own.  Every flag
// is cleared at the end.  The result is the same as rounds evaluated one level
// after another (the same-sequence lemma): the marks depend only on final counts.
//
// Pure rounds are skipped.  When round x ends with exactly its movers M climbing
// on (none stopped, nobody new marked), a following round y moves M from y to y+1
// and changes nothing else as long as no neighbour of M outside M sits on levels
// y .. y+2 (nobody left behind, nobody gaining an up- or up*-neighbour), no initial
// candidate sits on y+1 and every member still violates on y+1 (its up-degree is
// unchanged, so this holds while the cutoff stays below M's smallest up-degree).
// The scan of round x finds the lowest level >= x+1 of a non-mover neighbour and
// the climbing movers' smallest up-degree, so the team can run the next j pure
// rounds at once: the level jumps by j, and rounds, moves and visits are counted
// as the j rounds would have counted them.  The members' level words still read
// x+1 (with their flag) until their next scan rewrites them; readers of that scan
// take a flagged word anywhere from x+1 up as a mover (lmo = x+1), and j is even so
// that the flag's parity is the one of the new level.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t level_flag(int32_t l) { return (l & 1) ? kFlagOdd : kFlagEven; }

// Effects of a mover of level l on 16 neighbours ws (level words lv), in two
// passes so that the counter atomics of all 16 are in flight together: first every
// neighbour is classified and its counter updated -- a neighbour on l + 1 gains an
// up-neighbour (returning add: the one add that sees the old value equal to the
// cutoff marks it), one on l + 2 an up*-neighbour -- then the marks are set.
// Per slot q: bit q of push if the neighbour became a mover of level l + 1 here,
// of keep if it stays on level l + 1 or above after the round (an entry of the
// mover's up-list for its next move); aff counts neighbours whose counters
// changed; cnt4[q / 4] counts the neighbours left on l; low gets the lowest level
// above l of a neighbour that is no mover.  Movers of l read as flagged words on
// levels lmo .. l + 1 (lmo = l unless pure rounds were just skipped).
__device__ __forceinline__ void ins_effects16(const GraphCtx &g, const int32_t (&ws)[16], const int32_t (&lv)[16],
                                              int32_t l, int32_t lmo, int32_t fcur, int32_t fnext, int32_t cut_next,
                                              int (&cnt4)[4], int32_t &low, unsigned &push, unsigned &keep,
                                              unsigned &aff) {
    int32_t old[16];
    unsigned a1m = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int32_t w = ws[q], raw = lv[q], f = raw & kLevelMask;
        const bool ok = valid_id(g, w);  // not an empty slot or a tombstone
        const bool mov = ok && (raw & fcur) && f >= lmo && f <= l + 1;  // a mover of level l as well
        const bool other = ok && !mov;
        cnt4[q >> 2] += (other && f == l) ? 1 : 0;
        const bool above = other && f > l;
        if (above) low = min(low, f);
        const bool a1 = above && f == l + 1, a2 = above && f == l + 2;
        old[q] = 0;
        if (a1) old[q] = atomicAdd(&g.up[w], 1);
        if (a2) atomicAdd(&g.upstar[w], 1);
        a1m |= a1 ? 1u << q : 0u;
        keep |= (mov || above) ? 1u << q : 0u;
        aff += (a1 || a2) ? 1u : 0u;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q)
        if (((a1m >> q) & 1u) && old[q] == cut_next && !(atomicOr(&g.level[ws[q]], fnext) & fnext)) push |= 1u << q;
}

// A mover of level l whose whole table has been scanned (total = its neighbours
// left on l): new up* = old up (its neighbours on l or above), new up = old up -
// total, level l + 1; returns true if it violates Invariant 1 on l + 1 as well.
// old_up: the mover's up-degree, read at any time during the round (only this
// function writes it while the round runs).
__device__ __forceinline__ bool ins_finish_mover(const GraphCtx &g, int32_t v, int32_t old_up, int32_t total,
                                                 int32_t l, int32_t fcur, int32_t fnext, int32_t cut_next) {
    const int32_t nu = old_up - total;
    g.upstar[v] = old_up;
    g.up[v] = nu;
    const bool again = nu > cut_next;
    g.level[v] = (l + 1) | fcur | (again ? fnext : 0);
    return again;
}

// The lanes' movers that climb on (again): their new up-degrees and degrees go
// into the block's totals -- reduced over the warp first, then one lane's shared
// atomics (published once per block at the end of the phase).  All lanes call.
__device__ __forceinline__ void ff_note(const RoundStage &st, bool again, int32_t nu, int32_t deg) {
    const unsigned m = __ballot_sync(kFull, again);
    if (m == 0) return;
    const int32_t mn = (int32_t)__reduce_min_sync(kFull, again ? (unsigned)nu : (unsigned)kInf);
    const unsigned long long sd = warp_sum64(again ? (unsigned long long)deg : 0ull);
    const unsigned long long su = warp_sum64(again ? (unsigned long long)nu : 0ull);
    if (lane_id() == __ffs(m) - 1) {
        atomicAdd(&st.ff[0], __popc(m));
        atomicMin(&st.ff[1], mn);
        atomicAdd(&st.ff64[0], sd);
        atomicAdd(&st.ff64[1], su);
    }
}

// Queue the table scans of the lanes' newly marked vertices (their first move of
// the batch: up-list room for all their neighbours).
__device__ __forceinline__ void enqueue_marked(const GraphCtx &g, const RoundStage &st, bool mk, int32_t w,
                                               int k1, int32_t *wsm) {
    int32_t c = 0, d = 0;
    int64_t off = 0;
    if (mk) {
        c = g.cap[w];
        off = g.off[w];
        d = g.deg[w];
    }
    enqueue_ins(g, st, mk, w, c, off, -1, 0, d, k1, wsm);
}

// Marked neighbours wait in a per-warp buffer (kMarkCap ids in the warp's shared
// scratch, after the 160 ints enqueue_mover uses) and are queued 32 at a time, so
// their table lookups are issued together.
constexpr int kMarkCap = 256;

__device__ __forceinline__ void marks_flush(const GraphCtx &g, const RoundStage &st, int32_t *mbuf, int &mc,
                                            int k1, int32_t *wsm) {
    for (int b = 0; b < mc; b += 32) {
        const int i = b + lane_id();
        const bool mk = i < mc;
        enqueue_marked(g, st, mk, mk ? mbuf[i] : 0, k1, wsm);
    }
    __syncwarp();
    mc = 0;
}

// Append the lanes' marked neighbours (bits of push over ws); mc is warp-uniform.
__device__ __forceinline__ void marks_add(const GraphCtx &g, const RoundStage &st, unsigned push,
                                          const int32_t (&ws)[16], int32_t *mbuf, int &mc, int k1, int32_t *wsm) {
    int tot;
    const int ex = warp_exclusive(__popc(push), &tot);
    if (tot == 0) return;
    if (mc + tot > kMarkCap) marks_flush(g, st, mbuf, mc, k1, wsm);
    if (tot > kMarkCap) {  // more than the buffer holds: queue them one slot position at a time
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const bool mk = (push >> q) & 1u;
            if (__any_sync(kFull, mk)) enqueue_marked(g, st, mk, ws[q], k1, wsm);
        }
        return;
    }
    int pos = mc + ex;
#pragma unroll
    for (int q = 0; q < 16; ++q)
        if ((push >> q) & 1u) mbuf[pos++] = ws[q];
    __syncwarp();
    mc += tot;
}

// Test the initial candidates S[s_lo, s_hi) on level L against Invariant 1 (warp
// ranks rotated by rot, so that a small test runs on other warps than a scan).
template <class Team>
__device__ void ins_test_initial(Team &T, const GraphCtx &g, const RoundStage &st, int32_t s_lo, int32_t s_hi,
                                 int32_t L, int32_t cut, int32_t *wsm, int rot, int k1) {
    const int32_t fl = level_flag(L);
    const int rank = (T.srank() + rot) % T.nwarps();
    for (int i0 = s_lo + rank * 32; i0 < s_hi; i0 += T.nwarps() * 32) {
        const int i = i0 + lane_id();
        bool mk = false;
        int32_t v = 0;
        if (i < s_hi) {
            v = g.S[i];
            const int32_t raw = g.level[v];
            if ((raw & kLevelMask) != L) report(g, kErrInternal, 6, v, raw, L);
            else if (g.up[v] > cut) mk = !(atomicOr(&g.level[v], fl) & fl);
        }
        enqueue_marked(g, st, mk, v, k1, wsm);
    }
}

template <class Team>
__device__ bool ins_rounds(Team &T, const GraphCtx &g, const int32_t *sh_upmax, int32_t *wsm, RoundStage st) {
    unsigned long long visits = 0, scanned = 0, upv = 0;
    unsigned aff = 0;  // neighbours whose counters a move changed
    const int lane = lane_id();
    const int4 *pool4 = reinterpret_cast<const int4 *>(g.slots);
    const int32_t nlev = g.ctl->nlev;
    int32_t *mbuf = wsm + 160;
    int mc = 0;
    int spos = 0;
    int32_t l = nlev > 0 ? g.levlist[spos++] : 0;
    int32_t lmo = l;     // movers of l read as flagged words on levels lmo .. l + 1
    bool ffed = false;   // pure rounds were skipped just before this phase
    bool scan = false;  // this phase scans the movers of l (else it tests the initial candidates on l)
    for (int k = 0; nlev > 0; ++k) {
        if ((scan && l >= g.K - 1) || k > 2 * g.K + 4) {  // the top group is never violated
            if (T.leader()) report(g, kErrInternal, 5, l, k, 0);
            return false;
        }
        const int cur = k % 3, nxt = (k + 1) % 3, old = (k + 2) % 3;
        // up-lists: read from buffer old (written in phase k - 1), written to buffer
        // cur (room handed out in phase k - 1), room handed out now from buffer nxt
        const int32_t *lin = g.lbuf[old];
        int32_t *lwr = g.lbuf[cur];
        int32_t *fill_cur = g.lfill[k & 1];  // reset when this phase's movers were queued
        const uint64_t t_phase = (g.trace && T.leader()) ? global_ns() : 0;
        int32_t tlc = 0, clc = 0, m = 0;
        bool has_init = false;
        if (T.leader()) {  // the lists of phase k - 1 are done with; phase k + 1 fills them next
            g.ctl->itl[old] = 0;
            g.ctl->icl[old] = 0;
            g.ctl->imcnt[old] = 0;
            g.ctl->ltop[old] = 0;  // allocated from in phase k + 1 (its contents are read now)
            g.ctl->icont[old] = 0;
            g.ctl->iminup_c[old] = 0;
            g.ctl->ilow_c[old] = 0;
            g.ctl->isdeg[old] = 0;
            g.ctl->isup[old] = 0;
        }
        int32_t low = kInf;  // lowest level above l of a neighbour of a mover that is no mover
        st.tl.gcnt = &g.ctl->itl[nxt];
        st.tl.glist = g.TL[nxt];
        st.tl.gcap = g.n;
        st.cl.gcnt = &g.ctl->icl[nxt];
        st.cl.glist = g.CL[nxt];
        st.cl.gcap = g.clcap;
        if (!scan) {
            const int32_t s_lo = l == 0 ? 0 : g.bins[l - 1], s_hi = g.bins[l];
            ins_test_initial(T, g, st, s_lo, s_hi, l, sh_upmax[l / g.Lg], wsm, 0, k + 1);
        } else {
            // counts, next initial-candidate level and its range (fetched at a grid barrier)
            int32_t s_lo, s_hi;
            if constexpr (Team::kGrid) {
                m = st.phs[1];
                tlc = st.phs[2];
                clc = st.phs[3];
                has_init = st.phs[4] == l + 1;
                s_lo = st.phs[5];
                s_hi = st.phs[6];
                if (ffed && has_init) {  // fetched for the level before the skip
                    s_lo = g.bins[l];
                    s_hi = g.bins[l + 1];
                }
            } else {
                m = g.ctl->imcnt[cur];
                tlc = g.ctl->itl[cur];
                clc = g.ctl->icl[cur];
                has_init = spos < nlev && g.levlist[spos] == l + 1;
                s_lo = has_init ? g.bins[l] : 0;
                s_hi = has_init ? g.bins[l + 1] : 0;
            }
            if (T.leader()) {
                atomicAdd(&g.ctl->st[kStRounds], 1ull);
                atomicAdd(&g.ctl->st[kStMoves], (unsigned long long)m);
            }
            const int32_t fcur = level_flag(l), fnext = level_flag(l + 1);
            const int32_t cut_next = sh_upmax[(l + 1) / g.Lg];
            if (has_init)  // initial candidates on l + 1
                ins_test_initial(T, g, st, s_lo, s_hi, l + 1, cut_next, wsm, T.nwarps() / 2, k + 1);
            // thread-mode movers: up to 4 groups (16 slots) per pass, loads issued together
            for (int i0 = T.srank() * 32; i0 < tlc; i0 += T.nwarps() * 32) {
                const int i = i0 + lane;
                const int4 it = i < tlc ? g.TL[cur][i] : make_int4(0, 0, 0, 0);
                const bool have = i < tlc && item_ok(g, it, it.y);
                const int ng = have ? (1 << it.y) >> 2 : 0;
                const int32_t up_v = have ? g.up[it.x] : 0;  // issued with the slot loads
                const int maxg = (int)__reduce_max_sync(kFull, (unsigned)ng);
                int cnt_l = 0, ideg = 0;
                for (int j0 = 0; j0 < maxg; j0 += 4) {
                    int32_t ws[16], lv[16];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int4 s4 = j0 + j < ng ? pool4[it.z + j0 + j] : empty4();
                        ws[4 * j] = s4.x; ws[4 * j + 1] = s4.y; ws[4 * j + 2] = s4.z; ws[4 * j + 3] = s4.w;
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q) lv[q] = valid_id(g, ws[q]) ? g.level[ws[q]] : 0;
                    unsigned push = 0, keep = 0;
                    int c4[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int q = 0; q < 16; ++q) ideg += ws[q] >= 0;
                    ins_effects16(g, ws, lv, l, lmo, fcur, fnext, cut_next, c4, low, push, keep, aff);
                    cnt_l += c4[0] + c4[1] + c4[2] + c4[3];
                    scanned += 4 * (unsigned long long)max(0, min(4, ng - j0));
                    marks_add(g, st, push, ws, mbuf, mc, k + 1, wsm);
                }
                visits += ideg;
                upv += up_v;
                const bool again = have && ins_finish_mover(g, it.x, up_v, cnt_l, l, fcur, fnext, cut_next);
                ff_note(st, again, up_v - cnt_l, ideg);
                enqueue_ins(g, st, again, it.x, have ? 1 << it.y : 0, (int64_t)it.z * 4, -1, 0, 0, k + 1, wsm);
            }
            // chunk items: four per warp iteration, all loads of a step issued together;
            // taken from the last warp down, so that in a small round the warps
            // scanning thread-mode items and those scanning chunks are different ones
            const int crank = T.nwarps() - 1 - T.srank();
            const int4 *lin4 = reinterpret_cast<const int4 *>(lin);
            for (int c0 = crank; c0 < clc; c0 += 4 * T.nwarps()) {
                int4 it[4];
                bool ok[4], in[4];
                int32_t ws[16], lv[16];
                int32_t upl = 0, lol = -1, dgl = 0;  // lane u < 4: item u's vertex: up-degree, output up-list, degree
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int cu = c0 + u * T.nwarps();
                    it[u] = cu < clc ? ((Team::kGrid && cu == crank) ? st.ph4[threadIdx.x >> 5] : g.CL[cur][cu]) : make_int4(0, 0, 0, 0);
                    const bool lst = (it[u].y & 31) == 31;
                    ok[u] = cu < clc && (lst ? (it[u].x >= 0 && it[u].x < g.n && it[u].w >= 0 && it[u].z >= 0 &&
                                                (int64_t)it[u].z * 4 + it[u].w <= g.lcap)
                                             : item_ok(g, it[u], it[u].y & 31));
                    if (lane == u && ok[u]) {
                        upl = g.up[it[u].x];
                        lol = g.lout[it[u].x];
                        dgl = g.deg[it[u].x];
                    }
                    const int ng = lst ? (it[u].w + 3) >> 2 : (1 << (it[u].y & 31)) >> 2;
                    const int j = (it[u].y >> 5) * (kChunk / 4) + lane;
                    in[u] = ok[u] && j < ng;
                    const int4 s4 = in[u] ? (lst ? lin4[it[u].z + j] : pool4[it[u].z + j]) : empty4();
                    ws[4 * u] = s4.x; ws[4 * u + 1] = s4.y; ws[4 * u + 2] = s4.z; ws[4 * u + 3] = s4.w;
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) lv[q] = valid_id(g, ws[q]) ? g.level[ws[q]] : 0;
                int cl4[4] = {0, 0, 0, 0};
                unsigned push = 0, keep = 0;
                ins_effects16(g, ws, lv, l, lmo, fcur, fnext, cut_next, cl4, low, push, keep, aff);
#pragma unroll
                for (int u = 0; u < 4; ++u) scanned += in[u] ? 4 : 0;
                marks_add(g, st, push, ws, mbuf, mc, k + 1, wsm);
                // per item u: neighbours left on l (cnt), entries kept for the up-list
                // (kept, with this lane's offset kex[u]); lane u < 4 then issues item u's
                // two atomics together: room in the up-list, and the chunk count
                int kex[4];
                int myc = 0, mykt = 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = warp_sum(cl4[u]);
                    int kt;
                    kex[u] = warp_exclusive(__popc((keep >> (4 * u)) & 0xFu), &kt);
                    if (lane == u) {
                        myc = c;
                        mykt = kt;
                    }
                }
                int4 mine = it[0];
                bool mok = ok[0];
#pragma unroll
                for (int u = 1; u < 4; ++u)
                    if (lane == u) {
                        mine = it[u];
                        mok = ok[u];
                    }
                const bool mlst = (mine.y & 31) == 31;
                int fbase = 0;
                bool last = false;
                int32_t total = 0;
                if (lane < 4 && mok) {
                    if (lol >= 0 && mykt > 0) fbase = atomicAdd(&fill_cur[mine.x], mykt);
                    const int nch = mlst ? max(1, (mine.w + kChunk - 1) / kChunk) : max(1, (1 << (mine.y & 31)) / kChunk);
                    last = true;
                    total = myc;
                    if (nch > 1) {
                        const unsigned long long o =
                            atomicAdd(&g.acc[mine.x], (1ull << 32) | (unsigned long long)(uint32_t)myc);
                        last = (int)(o >> 32) + 1 == nch;
                        total = (int32_t)(uint32_t)(o & 0xffffffffull) + myc;
                        if (last) g.acc[mine.x] = 0ull;
                    }
                }
                // the kept neighbours go to their mover's up-list
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t lo = __shfl_sync(kFull, lol, u);
                    const int kb0 = __shfl_sync(kFull, fbase, u);
                    if (lo < 0) continue;  // warp-uniform
                    const unsigned kb = (keep >> (4 * u)) & 0xFu;
                    int32_t *dst = lwr + (int64_t)lo * 4 + kb0 + kex[u];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if ((kb >> q) & 1u) *dst++ = ws[4 * u + q];
                }
                // the last chunk of a mover to finish completes it (lane u: item u)
                int32_t nul = 0;  // lane u < 4: item u's new up-degree
                bool cont = false;
                if (last) {
                    visits += dgl;  // a move examines the mover's neighbours: its degree
                    upv += upl;
                    nul = upl - total;
                    cont = ins_finish_mover(g, mine.x, upl, total, l, fcur, fnext, cut_next);
                    for (int p = nul; cont && lol >= 0 && (p & 3); ++p) lwr[(int64_t)lol * 4 + p] = kEmpty;
                }
                ff_note(st, cont, nul, dgl);
                // a mover that keeps climbing is scanned next from its up-list, or from
                // its table again when its list did not fit
                int32_t mc_cap = 0;
                int64_t moff = 0;
                if (cont && lol < 0) {
                    if (mlst) {
                        mc_cap = g.cap[mine.x];
                        moff = g.off[mine.x];
                    } else {
                        mc_cap = 1 << (mine.y & 31);
                        moff = (int64_t)mine.z * 4;
                    }
                }
                enqueue_ins(g, st, cont, mine.x, mc_cap, moff, (cont && lol >= 0) ? nul : -1, lol, nul, k + 1, wsm);
            }
            marks_flush(g, st, mbuf, mc, k + 1, wsm);
            low = (int32_t)__reduce_min_sync(kFull, (unsigned)low);
            if (lane == 0 && low < kInf) atomicMin(&st.ff[2], low);
        }
        const uint64_t t_work = (g.trace && T.leader()) ? global_ns() : 0;
        if (g.trace) {  // every block: when it finished its share of the phase
            __syncthreads();
            if (threadIdx.x == 0) {
                const unsigned long long tb = global_ns();
                atomicMax(&g.ctl->tw_max[k & 1], tb);
                atomicMax(&g.ctl->tw_min_c[k & 1], ~tb);
            }
        }
        stage_flush_round(g, st, 6u);
        if (threadIdx.x == 0) {
            if (*st.movers) {
                atomicAdd(&g.ctl->imcnt[nxt], *st.movers);
                *st.movers = 0;
            }
            if (st.ff[0]) {  // the block's climbing movers (complements: zero means none)
                atomicAdd(&g.ctl->icont[nxt], st.ff[0]);
                atomicMax(&g.ctl->iminup_c[nxt], kInf - st.ff[1]);
                atomicAdd(&g.ctl->isdeg[nxt], st.ff64[0]);
                atomicAdd(&g.ctl->isup[nxt], st.ff64[1]);
                st.ff[0] = 0;
                st.ff[1] = kInf;
                st.ff64[0] = 0;
                st.ff64[1] = 0;
            }
            if (st.ff[2] < kInf) {
                atomicMax(&g.ctl->ilow_c[nxt], kInf - st.ff[2]);
                st.ff[2] = kInf;
            }
        }
        // the level the next phase scans if it has movers, and its initial-candidate
        // entry; warp 0 fetches them with the next phase's counts and each warp's
        // first chunk item while it passes the barrier
        int spos2 = spos;
        int32_t l2 = l;
        if (scan) {
            if (has_init) ++spos2;
            ++l2;
        }
        bool passed;
        if constexpr (Team::kGrid) {
            const int4 *cl_next = g.CL[nxt];
            passed = T.sync_fetch(
                [&](int ln) {
                    if (ln < (int)(blockDim.x >> 5)) {  // warp ln of the block: its first chunk item
                        const int cr = T.nwarps() - 1 - (ln * T.nblocks() + T.bid());  // warp ln's srank
                        st.ph4[ln] = cr < g.clcap ? cl_next[cr] : make_int4(0, 0, 0, 0);
                    } else if (ln == 16) {
                        st.phs[1] = g.ctl->imcnt[nxt];
                    } else if (ln == 17) {
                        st.phs[2] = g.ctl->itl[nxt];
                    } else if (ln == 18) {
                        st.phs[3] = g.ctl->icl[nxt];
                    } else if (ln == 19) {
                        st.phs[4] = spos2 < nlev ? g.levlist[spos2] : kInf;
                    } else if (ln == 20) {
                        st.phs[5] = l2 < g.K ? g.bins[l2] : 0;
                    } else if (ln == 21) {
                        st.phs[6] = l2 < g.K ? g.bins[l2 + 1] : 0;
                    } else if (ln == 22) {
                        st.phs[7] = g.ctl->icont[nxt];
                    } else if (ln == 23) {
                        st.phs[8] = g.ctl->ilow_c[nxt];
                    } else if (ln == 24) {
                        st.phs[9] = g.ctl->iminup_c[nxt];
                    }
                },
                st.phs);
        } else {
            passed = T.sync();
        }
        if (!passed) return false;
        // the next phase: the movers of l + 1 (after a scan) or of l (after a test),
        // else the initial candidates of the next level that has some
        spos = spos2;
        l = l2;
        lmo = l;
        ffed = false;
        const int32_t nm = Team::kGrid ? st.phs[1] : g.ctl->imcnt[nxt];
        int32_t skip = 0;
        if (scan && m > 0 && nm == m) {
            const int32_t ncont = Team::kGrid ? st.phs[7] : g.ctl->icont[nxt];
            if (ncont == m) {  // the same movers climb on to l: skip the pure rounds ahead
                const int32_t lowc = Team::kGrid ? st.phs[8] : g.ctl->ilow_c[nxt];
                const int32_t mupc = Team::kGrid ? st.phs[9] : g.ctl->iminup_c[nxt];
                const int64_t low_lvl = lowc ? (int64_t)(kInf - lowc) : (int64_t)kInf;
                const int32_t minup = kInf - mupc;
                const int64_t init_lvl = spos < nlev ? (int64_t)(Team::kGrid ? st.phs[4] : g.levlist[spos]) : (int64_t)kInf;
                int gg = l / g.Lg;  // highest group whose cutoff stays below the smallest up-degree
                while (gg + 1 < g.G && sh_upmax[gg + 1] < minup) ++gg;
                const int64_t top = (int64_t)(gg + 1) * g.Lg - 1;
                // round l - 1 just ran; rounds l .. l + j - 1 are pure while no other
                // neighbour sits on l .. l + j + 1, no initial candidate on l + 1 .. l + j
                // and every member still violates on l + j
                int64_t j = min(min(low_lvl - l - 2, init_lvl - l - 1), top - l);
                j &= ~(int64_t)1;  // even: the movers' flag keeps its parity
                if (j >= 2) {
                    skip = (int32_t)j;
                    if (T.leader()) {
                        const unsigned long long jm = (unsigned long long)j * (unsigned long long)m;
                        const unsigned long long jv = (unsigned long long)j * g.ctl->isdeg[nxt];
                        const unsigned long long ju = (unsigned long long)j * g.ctl->isup[nxt];
                        atomicAdd(&g.ctl->st[kStRounds], (unsigned long long)j);
                        atomicAdd(&g.ctl->st[kStMoves], jm);
                        atomicAdd(&g.ctl->st[kStVisits], jv);
                        atomicAdd(&g.ctl->st[kStUpVisits], ju);
                        atomicAdd(&g.ctl->st[kStSkipRounds], (unsigned long long)j);
                        atomicAdd(&g.ctl->st[kStSkipMoves], jm);
                        atomicAdd(&g.ctl->st[kStSkipVisits], jv);
                        atomicAdd(&g.ctl->st[kStSkipUpVisits], ju);
                    }
                    lmo = l;
                    l += skip;
                    ffed = true;
                }
            }
        }
        if (g.trace && T.leader() && g.ctl->trace_n < g.trace_cap) {
            int32_t *rec = g.trace + 12 * g.ctl->trace_n++;
            const uint64_t t_end = global_ns();
            rec[0] = scan ? l2 - 1 : l2; rec[1] = scan ? 1 : 0; rec[2] = m; rec[3] = tlc; rec[4] = clc;
            rec[5] = (int32_t)(t_work - t_phase); rec[6] = (int32_t)(t_end - t_work);
            rec[7] = skip;
            // blocks' work ends after the phase start: the latest and the earliest
            rec[8] = (int32_t)(g.ctl->tw_max[k & 1] - t_phase);
            rec[9] = (int32_t)(~g.ctl->tw_min_c[k & 1] - t_phase);
            rec[10] = rec[11] = 0;
            g.ctl->tw_max[k & 1] = 0;
            g.ctl->tw_min_c[k & 1] = 0;
        }
        if (nm > 0) {
            scan = true;
            continue;
        }
        if (spos >= nlev) break;
        l = g.levlist[spos++];
        scan = false;
    }
    // clear the movers' flags (every vertex: flags sit only on vertices that moved)
    for (int64_t v = T.tid(); v < g.n; v += T.nthreads()) {
        const int32_t raw = g.level[v];
        if (raw & ~kLevelMask) g.level[v] = raw & kLevelMask;
    }
    visits = warp_sum64(visits);
    scanned = warp_sum64(scanned);
    upv = warp_sum64(upv);
    const unsigned long long affs = warp_sum64(aff);
    if (lane == 0) {
        atomicAdd(&g.ctl->st[kStVisits], visits);
        atomicAdd(&g.ctl->st[kStSlotsScanned], scanned);
        atomicAdd(&g.ctl->st[kStUpVisits], upv);
        if (affs) atomicAdd(&g.ctl->st[kStAffected], affs);
    }
    return T.sync();
}

// ---------------------------------------------------------------------------
// Step A5: desire-level.
//
// dl(w) for w on level lw violating Invariant 2 is the largest x <= lw-2 with
// cnt(x) >= dnmin[gn(x)], plus one, where cnt(x) is the number of neighbours on
// levels >= x; 0 if there is none.  The predicate is monotone in x (cnt falls,
// dnmin[gn(x)] rises), so the group that holds the answer is the highest group
// whose first level satisfies it (pass 1: per-group counts) and the level inside
// it comes from a per-level histogram of that group (pass 2, 256-level windows).
// One warp computes it for a small table, a whole block for a large one.
// ---------------------------------------------------------------------------

// Highest group k <= gmax whose first level satisfies the predicate, given the
// per-group neighbour counts hist[0..G); -1 if none.  One warp.
__device__ __forceinline__ int warp_best_group(const int32_t *hist, int G, int gmax, const int32_t *sh_dnmin) {
    const int lane = lane_id();
    const int per = (G + 31) / 32;  // groups per lane, lane 0 holds the lowest
    int local = 0;
    for (int b = 0; b < per; ++b) {
        const int k = lane * per + b;
        if (k < G) local += hist[k];
    }
    // suffix over lanes: neighbours in groups above this lane's range
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_down_sync(kFull, incl, o);
        if (lane + o < 32) incl += y;
    }
    int run = incl - local;
    int best = -1;
    for (int b = per - 1; b >= 0; --b) {
        const int k = lane * per + b;
        if (k < G) {
            run += hist[k];  // run = cnt(k * Lg)
            if (k <= gmax && run >= sh_dnmin[k] && best < 0) best = k;
        }
    }
    return (int)__reduce_max_sync(kFull, (unsigned)(best + 1)) - 1;
}

// Largest x in [lo, hi] with above + sum_{y=x..hi} h[y-lo] >= need, or -1; *cnt gets
// that sum at x (the neighbours on x or above).  One warp.
__device__ __forceinline__ int warp_window_find(const int32_t *h, int lo, int hi, int above, int need,
                                                int *cnt) {
    const int lane = lane_id();
    const int top = hi - lo;  // lane L covers offsets top-8L .. top-8L-7 (highest levels first)
    int local = 0;
    for (int b = 0; b < 8; ++b) {
        const int idx = top - 8 * lane - b;
        if (idx >= 0) local += h[idx];
    }
    int tot;
    int run = above + warp_exclusive(local, &tot);
    int found = -1, fcnt = 0;
    for (int b = 0; b < 8; ++b) {
        const int idx = top - 8 * lane - b;
        if (idx >= 0 && found < 0) {
            run += h[idx];
            if (run >= need) {
                found = lo + idx;
                fcnt = run;
            }
        }
    }
    const unsigned m = __ballot_sync(kFull, found >= 0);
    *cnt = m ? __shfl_sync(kFull, fcnt, __ffs(m) - 1) : 0;
    return m ? __shfl_sync(kFull, found, __ffs(m) - 1) : -1;
}

// The levels of the neighbours in table t4[0..ng) seen by one lane of a warp or one
// thread of a block (groups start, start + stride, ...), four 4-slot groups per step
// so that 16 level loads are in flight: f(level) for every neighbour.
template <class F>
__device__ __forceinline__ void scan_levels(const GraphCtx &g, const int4 *t4, int32_t ng, int start, int stride,
                                            F f) {
    for (int j0 = start; j0 < ng; j0 += 4 * stride) {
        int32_t ws[16], lv[16];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u * stride;
            const int4 q = j < ng ? t4[j] : empty4();
            ws[4 * u] = q.x; ws[4 * u + 1] = q.y; ws[4 * u + 2] = q.z; ws[4 * u + 3] = q.w;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) lv[k] = ws[k] >= 0 ? g.level[ws[k]] : -1;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (lv[k] >= 0) f(lv[k]);
    }
}

// Sum of h[lo..hi] (at most 256 entries) over a warp.
__device__ __forceinline__ int warp_range_sum(const int32_t *h, int lo, int hi) {
    int s = 0;
    for (int k = lo + lane_id(); k <= hi; k += 32) s += h[k];
    return warp_sum(s);
}

// Desire-level of w on level lw (Definition): the largest l' < lw whose level below
// has at least dnmin[gn(l'-1)] neighbours on it or above, found from a histogram of
// the neighbours' groups and then of the levels in the best group.  The first scan
// also counts the 256 levels just below lw - 1 one by one: when the best group lies
// in that window (the common case) no second scan is needed.  *slack gets, for an
// answer d > 0, the neighbours on d - 1 or above minus dnmin[gn(d - 1)] (>= 0; kInf
// for d = 0, 0 where it is not counted): while later moves do not take it below 0,
// the answer stays d.
__device__ int32_t warp_desire_level(const GraphCtx &g, int32_t w, int32_t lw, const int32_t *sh_dnmin,
                                     int32_t *hist, int32_t *slack) {
    *slack = kInf;
    if (lw < 2) return 0;
    const int lane = lane_id();
    const int32_t Lg = g.Lg, G = g.G;
    const int32_t ng = g.cap[w] >> 2;
    const int4 *t4 = reinterpret_cast<const int4 *>(g.slots + g.off[w]);
    const int32_t xmax = lw - 2;
    if (ng <= 128) {
        // The whole table in registers (four 16-byte groups per lane): the answer by
        // bisection on the definition's predicate P(x) = cnt(x) >= dnmin[gn(x)],
        // which holds for every x up to the answer's level and for none above (cnt
        // does not rise with x, dnmin does not fall), each cnt(x) one warp sum.
        int32_t lvv[16];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = lane + 32 * u;
            const int4 q = j < ng ? t4[j] : empty4();
            lvv[4 * u] = q.x >= 0 ? g.level[q.x] : -1;
            lvv[4 * u + 1] = q.y >= 0 ? g.level[q.y] : -1;
            lvv[4 * u + 2] = q.z >= 0 ? g.level[q.z] : -1;
            lvv[4 * u + 3] = q.w >= 0 ? g.level[q.w] : -1;
        }
        auto cnt_ge = [&](int32_t x) {
            int c = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) c += lvv[k] >= x ? 1 : 0;
            return (int32_t)__reduce_add_sync(kFull, (unsigned)c);
        };
        if (cnt_ge(0) < sh_dnmin[0]) return 0;
        int32_t lo = 0, hi = xmax + 1;  // P(lo) holds; P(hi) is taken as false
        while (hi - lo > 1) {
            const int32_t mid = lo + ((hi - lo) >> 1);
            if (cnt_ge(mid) >= sh_dnmin[mid / Lg]) lo = mid;
            else hi = mid;
        }
        *slack = cnt_ge(lo) - sh_dnmin[lo / Lg];
        return lo + 1;
    }
    const int32_t w0 = max(0, xmax - (kWindow - 1));
    int32_t *win = hist + G;  // levels w0..xmax one by one, win[kWindow]: above xmax
    const bool one = G + kWindow + 1 <= kWarpHist;
    for (int k = lane; k < G; k += 32) hist[k] = 0;
    if (one)
        for (int k = lane; k <= kWindow; k += 32) win[k] = 0;
    __syncwarp();
    if (one) {
        scan_levels(g, t4, ng, lane, 32, [&](int32_t x) {
            atomicAdd(&hist[x / Lg], 1);
            if (x > xmax) atomicAdd(&win[kWindow], 1);
            else if (x >= w0) atomicAdd(&win[x - w0], 1);
        });
    } else {
        scan_levels(g, t4, ng, lane, 32, [&](int32_t x) { atomicAdd(&hist[x / Lg], 1); });
    }
    __syncwarp();
    const int best = warp_best_group(hist, G, xmax / Lg, sh_dnmin);
    __syncwarp();
    if (best < 0) return 0;
    const int32_t need = sh_dnmin[best], a = best * Lg;
    int32_t hi = min((best + 1) * Lg - 1, xmax);
    int cnt = 0;
    *slack = 0;
    if (one && a >= w0) {  // the best group's levels were counted by the first scan
        const int above = win[kWindow] + warp_range_sum(win, hi + 1 - w0, xmax - w0);
        const int found = warp_window_find(win + (a - w0), a, hi, above, need, &cnt);
        if (found >= 0) *slack = cnt - need;
        return found >= 0 ? found + 1 : a + 1;  // a + 1 unreachable: cnt(a) >= need holds
    }
    for (;;) {
        const int32_t lo = max(a, hi - (kWindow - 1));
        __syncwarp();
        for (int k = lane; k < kWindow + 1; k += 32) hist[k] = 0;
        __syncwarp();
        scan_levels(g, t4, ng, lane, 32, [&](int32_t x) {
            if (x > hi) atomicAdd(&hist[kWindow], 1);
            else if (x >= lo) atomicAdd(&hist[x - lo], 1);
        });
        __syncwarp();
        const int found = warp_window_find(hist, lo, hi, hist[kWindow], need, &cnt);
        __syncwarp();
        if (found >= 0) {
            *slack = cnt - need;
            return found + 1;
        }
        if (lo == a) return a + 1;  // unreachable: cnt(a) >= need holds
        hi = lo - 1;
    }
}

__device__ int32_t block_desire_level(const GraphCtx &g, int32_t w, int32_t lw, const int32_t *sh_dnmin,
                                      int32_t *hist, int32_t *res, int32_t *slack) {
    *slack = kInf;  // as in warp_desire_level
    if (lw < 2) return 0;
    const int32_t Lg = g.Lg, G = g.G;
    const int32_t ng = g.cap[w] >> 2;
    const int4 *t4 = reinterpret_cast<const int4 *>(g.slots + g.off[w]);
    const int32_t xmax = lw - 2;
    const int32_t w0 = max(0, xmax - (kWindow - 1));
    int32_t *win = hist + G;  // as in warp_desire_level: one scan when the answer is near
    const bool one = G + kWindow + 1 <= kWarpHist;
    for (int k = threadIdx.x; k < G; k += blockDim.x) hist[k] = 0;
    if (one)
        for (int k = threadIdx.x; k <= kWindow; k += blockDim.x) win[k] = 0;
    __syncthreads();
    if (one) {
        scan_levels(g, t4, ng, threadIdx.x, blockDim.x, [&](int32_t x) {
            atomicAdd(&hist[x / Lg], 1);
            if (x > xmax) atomicAdd(&win[kWindow], 1);
            else if (x >= w0) atomicAdd(&win[x - w0], 1);
        });
    } else {
        scan_levels(g, t4, ng, threadIdx.x, blockDim.x, [&](int32_t x) { atomicAdd(&hist[x / Lg], 1); });
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int best = warp_best_group(hist, G, xmax / Lg, sh_dnmin);
        if (threadIdx.x == 0) *res = best;
    }
    __syncthreads();
    const int best = *res;
    __syncthreads();
    if (best < 0) return 0;
    const int32_t need = sh_dnmin[best], a = best * Lg;
    int32_t hi = min((best + 1) * Lg - 1, xmax);
    *slack = 0;
    if (one && a >= w0) {  // the best group's levels were counted by the first scan
        if (threadIdx.x < 32) {
            int cnt = 0;
            const int above = win[kWindow] + warp_range_sum(win, hi + 1 - w0, xmax - w0);
            const int found = warp_window_find(win + (a - w0), a, hi, above, need, &cnt);
            if (threadIdx.x == 0) {
                res[0] = found;
                res[1] = cnt;
            }
        }
        __syncthreads();
        const int found = res[0];
        if (found >= 0) *slack = res[1] - need;
        __syncthreads();
        return found >= 0 ? found + 1 : a + 1;  // a + 1 unreachable: cnt(a) >= need holds
    }
    for (;;) {
        const int32_t lo = max(a, hi - (kWindow - 1));
        for (int k = threadIdx.x; k < kWindow + 1; k += blockDim.x) hist[k] = 0;
        __syncthreads();
        scan_levels(g, t4, ng, threadIdx.x, blockDim.x, [&](int32_t x) {
            if (x > hi) atomicAdd(&hist[kWindow], 1);
            else if (x >= lo) atomicAdd(&hist[x - lo], 1);
        });
        __syncthreads();
        if (threadIdx.x < 32) {
            int cnt = 0;
            const int found = warp_window_find(hist, lo, hi, hist[kWindow], need, &cnt);
            if (threadIdx.x == 0) {
                res[0] = found;
                res[1] = cnt;
            }
        }
        __syncthreads();
        const int found = res[0];
        const int cntf = res[1];
        __syncthreads();
        if (found >= 0) {
            *slack = cntf - need;
            return found + 1;
        }
        if (lo == a) return a + 1;  // unreachable: cnt(a) >= need holds
        hi = lo - 1;
    }
}

// Desire-level of a vertex whose table has at most kThreadDl slots, by one thread:
// its neighbours' levels in registers, bisection on P(x) = cnt(x) >= dnmin[gn(x)]
// as in warp_desire_level.
constexpr int kThreadDl = 32;

__device__ __forceinline__ int32_t thread_desire_level(const GraphCtx &g, int32_t w, int32_t lw, int32_t c,
                                                       const int32_t *sh_dnmin, int32_t *slack) {
    *slack = kInf;
    if (lw < 2) return 0;
    const int4 *t4 = reinterpret_cast<const int4 *>(g.slots + g.off[w]);
    const int ng = c >> 2;
    int32_t lvv[kThreadDl];
#pragma unroll
    for (int u = 0; u < kThreadDl / 4; ++u) {
        const int4 q = u < ng ? t4[u] : empty4();
        lvv[4 * u] = q.x >= 0 ? g.level[q.x] : -1;
        lvv[4 * u + 1] = q.y >= 0 ? g.level[q.y] : -1;
        lvv[4 * u + 2] = q.z >= 0 ? g.level[q.z] : -1;
        lvv[4 * u + 3] = q.w >= 0 ? g.level[q.w] : -1;
    }
    auto cnt_ge = [&](int32_t x) {
        int32_t n = 0;
#pragma unroll
        for (int k = 0; k < kThreadDl; ++k) n += lvv[k] >= x ? 1 : 0;
        return n;
    };
    if (cnt_ge(0) < sh_dnmin[0]) return 0;
    int32_t lo = 0, hi = lw - 1;  // P(lo) holds; P(hi) is taken as false (answers stop at lw - 2)
    while (hi - lo > 1) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (cnt_ge(mid) >= sh_dnmin[mid / g.Lg]) lo = mid;
        else hi = mid;
    }
    *slack = cnt_ge(lo) - sh_dnmin[lo / g.Lg];
    return lo + 1;
}

// A desire-level d computed for w (slack sl): recorded, and a pending entry in
// P[q] unless it equals w's current pending level.
__device__ __forceinline__ void dl_record(const GraphCtx &g, int32_t w, int32_t d, int32_t sl, int q, int32_t lmin,
                                          int site) {
    g.dslack[w] = sl;
    if (d <= lmin) {
        report(g, kErrInternal, site, w, d, lmin);
    } else if (d != g.dlv[w]) {
        g.dlv[w] = d;
        const int pos = atomicAdd(&g.ctl->pcnt[q], 1);
        g.P[q][pos] = make_int4(w, d, 0, 0);
        atomicMin(&g.ctl->nextmin[q], d);
    }
}

// Desire-levels for every vertex of src[0..count) that violates Invariant 2
// (level > 0 and up* < dnmin[gn(level-1)]).  Two phases with a team barrier:
// classify into a warp list (small tables, from the front of RL) and a block list
// (large tables, from the back), then compute.  A result d becomes a pending
// entry in P[q] unless it equals the vertex's current pending level; results at
// or below lmin contradict the level lemma and are reported.  A pending vertex
// whose slack has not gone below 0 since its last evaluation would get the same
// answer again: that evaluation is counted (Algorithm 3 counts every evaluation)
// without the scan.
template <class Team>
__device__ bool dl_batch(Team &T, const GraphCtx &g, const int32_t *src, int32_t count, int q, int32_t lmin,
                         const int32_t *sh_dnmin, int32_t *whist, int32_t *bhist, unsigned long long &evals,
                         unsigned long long &evisits) {
    const int lane = lane_id();
    int32_t *RL = g.R[1];
    for (int i0 = T.srank() * 32; i0 < count; i0 += T.nwarps() * 32) {
        const int i = i0 + lane;
        bool viol = false, big = false;
        int32_t w = 0;
        if (i < count) {
            w = src[i];
            const int32_t lw = g.level[w], us = g.upstar[w], c = g.cap[w], dv = g.dlv[w];
            viol = lw > 0 && us < sh_dnmin[(lw - 1) / g.Lg];
            big = c > g.block_cap;
            if (viol && dv >= 0 && g.dslack[w] >= 0) {  // same answer as last time: counted only
                viol = false;
                evals++;
                evisits += g.deg[w];
            }
            if (viol && c <= kThreadDl) {  // a small table: this thread computes it
                viol = false;
                int32_t sl;
                const int32_t d = thread_desire_level(g, w, lw, c, sh_dnmin, &sl);
                evals++;
                evisits += g.deg[w];
                dl_record(g, w, d, sl, q, lmin, 10);
            }
        }
        const int pw = warp_append(&g.ctl->rcnt[1], viol && !big);
        if (viol && !big) RL[pw] = w;
        const int pb = warp_append(&g.ctl->rbcnt, viol && big);
        if (viol && big) RL[g.n - 1 - pb] = w;
    }
    if (!T.sync()) return false;
    const int32_t nw = g.ctl->rcnt[1], nb = g.ctl->rbcnt;
    for (int i = T.srank(); i < nw; i += T.nwarps()) {
        const int32_t w = RL[i], lw = g.level[w];
        int32_t sl;
        const int32_t d = warp_desire_level(g, w, lw, sh_dnmin, whist, &sl);
        if (lane == 0) {
            evals++;
            evisits += g.deg[w];
            dl_record(g, w, d, sl, q, lmin, 8);
        }
    }
    for (int i = T.bid(); i < nb; i += (T.nthreads() / blockDim.x)) {
        const int32_t w = RL[g.n - 1 - i], lw = g.level[w];
        int32_t sl;
        const int32_t d = block_desire_level(g, w, lw, sh_dnmin, bhist, bhist + kWarpHist, &sl);
        if (threadIdx.x == 0) {
            evals++;
            evisits += g.deg[w];
            dl_record(g, w, d, sl, q, lmin, 9);
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Step A6: deletion rounds (Algorithm 3).
// ---------------------------------------------------------------------------

// Effects of a mover (pv -> l) on neighbour w with level lw (w did not move if
// lw > l): v leaves Z_{lw} if lw <= pv and Z_{lw-1} if l < lw-1 <= pv.  The
// mover's own recount takes cu (neighbours >= l) and cs (>= l-1).  Returns 1 if
// w must be pushed for a desire-level recheck, 2 if that depends on w being
// pending (its dlv decides).
__device__ __forceinline__ int del_effect(const GraphCtx &g, int32_t w, int32_t lw, int32_t l, int32_t pv, int &cu,
                                          int &cs, unsigned &aff) {
    if (!valid_id(g, w)) return 0;
    cu += lw >= l;
    cs += lw >= l - 1;
    if (lw <= l) return 0;
    if (lw <= pv) atomicSub(&g.up[w], 1);
    if (lw - 1 > l && lw - 1 <= pv) atomicSub(&g.upstar[w], 1);
    aff += lw <= pv + 1;  // w lost an up- or up*-neighbour
    if (lw < l + 2) return 0;
    return lw - 1 <= pv ? 1 : 2;
}

// A mover (pv -> l) next to a pending vertex w whose desire-level is dv: the count
// behind w's answer (neighbours on dv - 1 or above) loses the mover when
// l < dv - 1 <= pv, and the slack of that answer with it.
__device__ __forceinline__ void del_slack(const GraphCtx &g, int32_t w, int32_t dv, int32_t l, int32_t pv) {
    const int32_t xs = dv - 1;
    if (l < xs && xs <= pv) atomicSub(&g.dslack[w], 1);
}

template <class Team>
__device__ bool del_rounds(Team &T, const GraphCtx &g, const int32_t stamp_base, const int32_t *sh_dnmin, int32_t *whist, int32_t *bhist,
                           int32_t *wsm, RoundStage st) {
    unsigned long long visits = 0, scanned = 0, evals = 0, evisits = 0;
    unsigned aff = 0;  // neighbours whose counters a move changed
    const int lane = lane_id();
    const int4 *pool4 = reinterpret_cast<const int4 *>(g.slots);
    for (int r = 0;; ++r) {
        const int p = r & 1, q = p ^ 1;
        const int32_t l = g.ctl->nextmin[p];
        if (l == kInf) break;
        if (r > g.K + 2) {
            if (T.leader()) report(g, kErrInternal, 7, l, r, 0);
            return false;
        }
        const int32_t sid = sid_of(stamp_base, l);
        const uint64_t t_round = (g.trace && T.leader()) ? global_ns() : 0;
        st.pk.gcnt = &g.ctl->pcnt[q];
        st.pk.glist = g.P[q];
        st.pk.gcap = 2 * (int64_t)g.n;
        st.tl.gcnt = &g.ctl->tlcnt[0];
        st.tl.glist = g.TL[0];
        st.tl.gcap = g.n;
        st.cl.gcnt = &g.ctl->clcnt[0];
        st.cl.glist = g.CL[0];
        st.cl.gcap = g.clcap;
        st.f.gcnt = &g.ctl->rcnt[0];
        st.f.glist = g.R[0];
        st.f.gcap = g.n;
        int32_t kmin = kInf;
        if (T.leader()) {
            g.ctl->rcnt[0] = 0;
            g.ctl->rcnt[1] = 0;
            g.ctl->rbcnt = 0;
        }
        // Phase 1: pending entries with dl == l move; the rest stay pending.
        const int32_t pc = g.ctl->pcnt[p];
        for (int i0 = T.srank() * 32; i0 < pc; i0 += T.nwarps() * 32) {
            const int i = i0 + lane;
            bool mover = false, keep = false;
            int32_t v = 0, d = 0, pv = 0, c = 0;
            int64_t off = 0;
            if (i < pc) {
                const int4 e = g.P[p][i];
                v = e.x;
                d = e.y;
                if (g.dlv[v] == d) {
                    if (d == l) {
                        mover = true;
                        pv = g.level[v];
                        c = g.cap[v];
                        off = g.off[v];
                        g.level[v] = l;
                        g.dlv[v] = -1;
                        g.up[v] = 0;
                        g.upstar[v] = 0;
                    } else {
                        keep = true;
                    }
                }
            }
            stage_push(st.pk, keep, make_int4(v, d, 0, 0));
            if (keep) kmin = min(kmin, d);
            enqueue_mover(g, st, mover, v, pv, c, off, wsm);
        }
        kmin = (int32_t)__reduce_min_sync(kFull, (unsigned)kmin);
        if (lane == 0 && kmin != kInf) atomicMin(st.bmin, kmin);
        stage_flush_round(g, st, 14u);
        if (threadIdx.x == 0) {
            if (*st.movers) atomicAdd(&g.ctl->mcnt[0], *st.movers);
            if (*st.bmin != kInf) atomicMin(&g.ctl->nextmin[q], *st.bmin);
            *st.movers = 0;
            *st.bmin = kInf;
        }
        if (!T.sync()) return false;
        // Phase 2: movers' neighbours.
        const uint64_t t_mid1 = (g.trace && T.leader()) ? global_ns() : 0;
        if (T.leader()) {
            const int32_t mc = g.ctl->mcnt[0];
            if (mc > 0) g.ctl->st[kStRounds] += 1;
            g.ctl->st[kStMoves] += (unsigned long long)mc;
            g.ctl->pcnt[p] = 0;
            g.ctl->nextmin[p] = kInf;
        }
        const int32_t tlc = g.ctl->tlcnt[0];
        for (int i0 = T.srank() * 32; i0 < tlc; i0 += T.nwarps() * 32) {
            const int i = i0 + lane;
            const int4 it = i < tlc ? g.TL[0][i] : make_int4(0, 0, 0, 0);
            const int ng = (i < tlc && item_ok(g, it, it.y)) ? (1 << it.y) >> 2 : 0;
            const int maxg = (int)__reduce_max_sync(kFull, (unsigned)ng);
            int cu = 0, cs = 0;
            for (int j0 = 0; j0 < maxg; j0 += 4) {
                int32_t ws[16], lv[16];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int4 s4 = j0 + j < ng ? pool4[it.z + j0 + j] : empty4();
                    ws[4 * j] = s4.x; ws[4 * j + 1] = s4.y; ws[4 * j + 2] = s4.z; ws[4 * j + 3] = s4.w;
                }
#pragma unroll
                for (int k = 0; k < 16; ++k) lv[k] = valid_id(g, ws[k]) ? g.level[ws[k]] : 0;
                unsigned push = 0, maybe = 0;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    visits += ws[k] >= 0;
                    const int e = del_effect(g, ws[k], lv[k], l, it.w, cu, cs, aff);
                    if (e == 1) push |= 1u << k;
                    if (e == 2) maybe |= 1u << k;
                }
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if ((push | maybe) >> k & 1u) {
                        const int32_t dv = g.dlv[ws[k]];
                        if (dv >= 0) {
                            push |= 1u << k;  // pending: rechecked
                            del_slack(g, ws[k], dv, l, it.w);
                        }
                    }
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if ((push >> k & 1u) && atomicExch(&g.stamp[ws[k]], sid) == sid) push &= ~(1u << k);
                scanned += 4 * (unsigned long long)max(0, min(4, ng - j0));
                stage_push_masked(st.f, push, ws);
            }
            if (i < tlc) {
                if (cu) atomicAdd(&g.up[it.x], cu);
                if (cs) atomicAdd(&g.upstar[it.x], cs);
            }
        }
        const int32_t clc = g.ctl->clcnt[0];
        for (int c0 = T.srank(); c0 < clc; c0 += 4 * T.nwarps()) {
            int4 it[4];
            bool in[4];
            int32_t ws[16], lv[16];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int cu = c0 + u * T.nwarps();
                it[u] = cu < clc ? g.CL[0][cu] : make_int4(0, 0, 0, 0);
                const int j = (it[u].y >> 5) * (kChunk / 4) + lane;
                in[u] = cu < clc && item_ok(g, it[u], it[u].y & 31) && j < ((1 << (it[u].y & 31)) >> 2);
                const int4 s4 = in[u] ? pool4[it[u].z + j] : empty4();
                ws[4 * u] = s4.x; ws[4 * u + 1] = s4.y; ws[4 * u + 2] = s4.z; ws[4 * u + 3] = s4.w;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) lv[k] = valid_id(g, ws[k]) ? g.level[ws[k]] : 0;
            int cu4[4] = {0, 0, 0, 0}, cs4[4] = {0, 0, 0, 0};
            unsigned push = 0, maybe = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                visits += ws[k] >= 0;
                const int e = del_effect(g, ws[k], lv[k], l, it[k >> 2].w, cu4[k >> 2], cs4[k >> 2], aff);
                if (e == 1) push |= 1u << k;
                if (e == 2) maybe |= 1u << k;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if ((push | maybe) >> k & 1u) {
                    const int32_t dv = g.dlv[ws[k]];
                    if (dv >= 0) {
                        push |= 1u << k;  // pending: rechecked
                        del_slack(g, ws[k], dv, l, it[k >> 2].w);
                    }
                }
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if ((push >> k & 1u) && atomicExch(&g.stamp[ws[k]], sid) == sid) push &= ~(1u << k);
#pragma unroll
            for (int u = 0; u < 4; ++u) scanned += in[u] ? 4 : 0;
            stage_push_masked(st.f, push, ws);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int a = warp_sum(cu4[u]), b = warp_sum(cs4[u]);
                if (lane == 0) {
                    if (a) atomicAdd(&g.up[it[u].x], a);
                    if (b) atomicAdd(&g.upstar[it[u].x], b);
                }
            }
        }
        stage_flush_round(g, st, 1u);
        if (!T.sync()) return false;
        // Phase 3: neighbours that now violate Invariant 2 get their desire-level
        // recomputed (it always lands above l).
        const uint64_t t_mid2 = (g.trace && T.leader()) ? global_ns() : 0;
        int32_t tr_movers = 0;
        if (g.trace && T.leader()) tr_movers = g.ctl->mcnt[0];
        if (T.leader()) {
            g.ctl->mcnt[0] = 0;
            g.ctl->tlcnt[0] = 0;
            g.ctl->clcnt[0] = 0;
        }
        if (!dl_batch(T, g, g.R[0], g.ctl->rcnt[0], q, l, sh_dnmin, whist, bhist, evals, evisits)) return false;
        if (!T.sync()) return false;
        if (g.trace && T.leader() && g.ctl->trace_n < g.trace_cap) {
            int32_t *rec = g.trace + 12 * g.ctl->trace_n++;
            const uint64_t t_end = global_ns();
            rec[0] = l; rec[1] = pc; rec[2] = tr_movers; rec[3] = tlc; rec[4] = clc;
            rec[5] = (int32_t)(t_mid1 - t_round); rec[6] = (int32_t)(t_mid2 - t_mid1);
            rec[7] = (int32_t)(t_end - t_mid2);
            rec[8] = g.ctl->rcnt[1];  // desire-levels computed by a warp after the classifying pass
            rec[9] = g.ctl->rbcnt;    // and by a block
            rec[10] = rec[11] = 0;
        }
    }
    visits = warp_sum64(visits);
    scanned = warp_sum64(scanned);
    const unsigned long long affs = warp_sum64(aff);
    if (lane == 0) {
        atomicAdd(&g.ctl->st[kStVisits], visits);
        atomicAdd(&g.ctl->st[kStSlotsScanned], scanned);
        if (affs) atomicAdd(&g.ctl->st[kStAffected], affs);
    }
    if (evals) {
        atomicAdd(&g.ctl->st[kStDlEvals], evals);
        atomicAdd(&g.ctl->st[kStDlVisits], evisits);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Insertion, jump variant (the implementation note of the Experiments section:
// a filter and sort computes a desire-level for the vertices moved up instead of
// moving them one level at a time).  Read as: each round takes the lowest level l
// that holds a violator of Invariant 1; every violator on l moves at once to its
// target, the lowest level above l on which it would satisfy Invariant 1 with
// every other vertex where it is (the other movers still on l).  Final levels
// equal Algorithm 2's (both reach the least assignment at or above the starting
// levels under which Invariant 1 holds everywhere); rounds and moves differ.
//
// Violators wait in a pending list {v, level} (each vertex at most once: a vertex
// is listed when it starts to violate and stays a violator until its round).
// Round r, three team barriers:
//   A: the previous round's movers lose their flag; the pending entries on l
//      become this round's movers (flag of r's parity in the level word, listed in
//      TL[r mod 3]), the others stay (marked in place; the list is rewritten once
//      most of it has been taken); then one warp per mover computes its target from
//      a histogram of its neighbours' levels above l (levels read before any move
//      of the round: the flags are masked), a block per large table; targets go to
//      dlv.
//   B: every mover scans its table once more: a neighbour that is a mover counts
//      at its target, any other at its level; a non-mover w on level lw gains an
//      up-neighbour if l < lw <= t and an up*-neighbour if l + 1 < lw <= t + 1, and
//      joins the pending list when that first takes its up-degree past its cutoff;
//      the mover's up and up* are recounted and it stays pending on t if it still
//      violates there.  The flag stays on until the next round's phase A, so every
//      reader of B tells movers from the rest.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t round_flag(int r) { return (r & 1) ? kFlagOdd : kFlagEven; }

// Smallest x in [lo, hi] (hi - lo < 256) with above + sum_{y=x..hi} h[y-lo] <= upmax
// of x's group, or -1.  The count falls and the bound rises with x, so the test
// fails below the answer and passes from it on.  One warp.
__device__ __forceinline__ int warp_jump_find(const int32_t *h, int lo, int hi, int above, int32_t Lg,
                                              const int32_t *sh_upmax) {
    const int lane = lane_id();
    int local = 0;  // lane L covers offsets 8L .. 8L+7, ascending
    for (int b = 0; b < 8; ++b)
        if (lo + 8 * lane + b <= hi) local += h[8 * lane + b];
    int incl = local;  // suffix over the lanes above
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_down_sync(kFull, incl, o);
        if (lane + o < 32) incl += y;
    }
    int run = above + incl - local;
    int found = -1;
    for (int b = 7; b >= 0; --b) {
        const int x = lo + 8 * lane + b;
        if (x <= hi) {
            run += h[8 * lane + b];  // run = neighbours on x or above
            if (run <= sh_upmax[x / Lg]) found = x;
        }
    }
    const unsigned m = __ballot_sync(kFull, found >= 0);
    return m ? __shfl_sync(kFull, found, __ffs(m) - 1) : -1;
}

// Target of a mover v of level l (warp, or whole block when blk): windows of 256
// levels from l + 1 up, one table scan each (the first almost always holds it).
template <bool blk>
__device__ int32_t jump_target(const GraphCtx &g, int32_t v, int32_t l, const int32_t *sh_upmax, int32_t *hist,
                               int32_t *res) {
    const int32_t ng = g.cap[v] >> 2;
    const int4 *t4 = reinterpret_cast<const int4 *>(g.slots + g.off[v]);
    const int start = blk ? (int)threadIdx.x : lane_id();
    const int stride = blk ? (int)blockDim.x : 32;
    for (int32_t lo = l + 1; lo < g.K; lo += kWindow) {
        const int32_t hi = min(lo + kWindow - 1, g.K - 1);
        for (int k = start; k <= kWindow; k += stride) hist[k] = 0;
        if (blk) __syncthreads(); else __syncwarp();
        scan_levels(g, t4, ng, start, stride, [&](int32_t raw) {
            const int32_t x = raw & kLevelMask;
            if (x > hi) atomicAdd(&hist[kWindow], 1);
            else if (x >= lo) atomicAdd(&hist[x - lo], 1);
        });
        if (blk) __syncthreads(); else __syncwarp();
        int found;
        if (blk) {
            if (threadIdx.x < 32) {
                const int f = warp_jump_find(hist, lo, hi, hist[kWindow], g.Lg, sh_upmax);
                if (threadIdx.x == 0) *res = f;
            }
            __syncthreads();
            found = *res;
            __syncthreads();
        } else {
            found = warp_jump_find(hist, lo, hi, hist[kWindow], g.Lg, sh_upmax);
            __syncwarp();
        }
        if (found >= 0) return found;
    }
    return g.K - 1;  // not reached: the top group's bound is n
}

// Append the lanes' {v, level} with pred to pending list pl (warp-collective) and
// fold their levels into the next round's minimum (slot ps); other: the entries are
// not movers of this round staying on the next level.
__device__ __forceinline__ void jump_push(const GraphCtx &g, int pl, int ps, bool pred, int32_t v, int32_t lv,
                                          bool other) {
    const int pos = warp_append(&g.ctl->jpend[pl], pred);
    if (pred) {
        if (pos < 2 * g.n) g.P[pl][pos] = make_int4(v, lv, 0, 0);
        else report(g, kErrListOverflow, 20, pos, v, lv);
    }
    const int32_t mn = (int32_t)__reduce_min_sync(kFull, pred ? (unsigned)lv : (unsigned)kInf);
    if (lane_id() == 0 && mn < kInf) {
        atomicMax(&g.ctl->jnext_c[ps], kInf - mn);
        if (other) atomicMax(&g.ctl->jother_c[ps], kInf - mn);
    }
}

// Phase B for one mover v (old level l, target tv, round flag flr): warp, or
// block when blk; new pending entries go to list pl, the round's totals to slot p.
// Returns its degree (visits); red: 4 ints of block scratch.
template <bool blk>
__device__ int32_t jump_apply(const GraphCtx &g, int32_t v, int32_t l, int32_t tv, int32_t flr, int pl, int p,
                              const int32_t *sh_upmax, int32_t *red, unsigned *aff) {
    const int32_t ng = g.cap[v] >> 2;
    const int4 *t4 = reinterpret_cast<const int4 *>(g.slots + g.off[v]);
    const int start = blk ? (int)threadIdx.x : lane_id();
    const int stride = blk ? (int)blockDim.x : 32;
    int cu = 0, cs = 0, dg = 0;
    int32_t low = kInf;  // lowest level above l of a neighbour that is no mover
    const int ng_iter = blk ? ((ng + stride - 1) / stride) * stride : ((ng + 31) & ~31);
    for (int j = start; j < ng_iter; j += stride) {  // every lane of a warp runs every step
        const int4 q = j < ng ? t4[j] : empty4();
        const int32_t ws[4] = {q.x, q.y, q.z, q.w};
        int32_t raw[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) raw[u] = valid_id(g, ws[u]) ? g.level[ws[u]] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            bool push = false;
            int32_t lw = 0;
            if (raw[u] >= 0) {
                ++dg;
                int32_t fw;
                if (raw[u] & flr) {
                    fw = g.dlv[ws[u]];  // a mover: counts at its target
                } else {
                    lw = raw[u] & kLevelMask;
                    fw = lw;
                    if (lw > l) low = min(low, lw);
                    if (l < lw && lw <= tv) push = atomicAdd(&g.up[ws[u]], 1) == sh_upmax[lw / g.Lg];
                    if (l + 1 < lw && lw <= tv + 1) atomicAdd(&g.upstar[ws[u]], 1);
                    *aff += l < lw && lw <= tv + 1;
                }
                cu += fw >= tv;
                cs += fw >= tv - 1;
            }
            if (__any_sync(kFull, push)) jump_push(g, pl, p, push, ws[u], lw, true);
        }
    }
    cu = warp_sum(cu);
    cs = warp_sum(cs);
    dg = warp_sum(dg);
    low = (int32_t)__reduce_min_sync(kFull, (unsigned)low);
    if (blk) {
        if (threadIdx.x == 0) {
            red[0] = red[1] = red[2] = 0;
            red[3] = kInf;
        }
        __syncthreads();
        if (lane_id() == 0) {
            atomicAdd(&red[0], cu);
            atomicAdd(&red[1], cs);
            atomicAdd(&red[2], dg);
            atomicMin(&red[3], low);
        }
        __syncthreads();
        cu = red[0];
        cs = red[1];
        dg = red[2];
        low = red[3];
        __syncthreads();
    }
    const bool lead = blk ? threadIdx.x < 32 : true;  // one warp finishes the mover
    if (lead) {
        const bool stay = cu > sh_upmax[tv / g.Lg];
        if (lane_id() == 0) {
            g.up[v] = cu;
            g.upstar[v] = cs;
            g.level[v] = tv | flr;  // still flagged: readers of this phase take dlv
            if (low < kInf) atomicMax(&g.ctl->jlow_c[p], kInf - low);
            if (tv != l + 1) atomicAdd(&g.ctl->jnonunit[p], 1);
            if (stay) {
                atomicAdd(&g.ctl->jstay[p], 1);
                atomicMax(&g.ctl->jminup_c[p], kInf - cu);
                atomicAdd(&g.ctl->jsdeg[p], (unsigned long long)dg);
            }
        }
        jump_push(g, pl, p, lane_id() == 0 && stay, v, tv, tv != l + 1);
    }
    return dg;
}

template <class Team>
__device__ bool ins_rounds_jump(Team &T, const GraphCtx &g, const int32_t *sh_upmax, int32_t *whist,
                                int32_t *sh_block) {
    const int lane = lane_id();
    const int32_t tc = g.ctl->tcount;
    int32_t *bmin = sh_block + kWarpHist + 16;  // block's lowest carried level
    if (threadIdx.x == 0) bmin[0] = kInf;
    // every endpoint of the batch that violates now is pending on its level
    for (int i0 = T.wid() * 32; i0 < tc; i0 += T.nwarps() * 32) {
        const int i = i0 + lane;
        bool v_ = false;
        int32_t x = 0, lx = 0;
        if (i < tc) {
            x = g.touched[i];
            g.inc[x] = 0;
            lx = g.level[x];
            v_ = g.up[x] > sh_upmax[lx / g.Lg];
        }
        jump_push(g, 0, 0, v_, x, lx, true);
    }
    if (!T.sync()) return false;
    unsigned long long visits = 0;
    unsigned aff = 0;    // neighbours whose counters a move changed
    int pb = 0;          // the pending list in use (entries taken are marked in place)
    int32_t lprev = -1;  // level of the previous round
    int r = 0;
    for (;; ++r) {
        const int cur = r & 1, nxt = cur ^ 1;  // slots of this round's and the next round's totals
        const int32_t nc = g.ctl->jnext_c[cur];
        if (nc == 0) break;
        int32_t l = kInf - nc;
        // Pure rounds (as for Algorithm 2's rounds): when every mover of the previous
        // round (level x) went to x + 1 and still violates there, nothing else is
        // pending on x + 1, and no neighbour of theirs outside them sits on x + 1 ..
        // x + j + 2, each of the next j rounds moves the same set up one level (its
        // members' targets stay at the next level: their count above it is their
        // outside neighbours, all higher, within the cutoff that already held) and
        // changes nothing else, while no other entry is pending on those levels and the
        // cutoff stays below their smallest up-degree.  Those rounds are counted, not run.
        int32_t skip = 0;
        if (r > 0 && l == lprev + 1) {
            const int32_t mprev_n = g.ctl->jmov[(r + 2) % 3];
            if (g.ctl->jstay[cur] == mprev_n && g.ctl->jnonunit[cur] == 0) {
                const int32_t oc = g.ctl->jother_c[cur], lc = g.ctl->jlow_c[cur];
                const int64_t other = oc ? (int64_t)(kInf - oc) : (int64_t)kInf;
                const int64_t low = lc ? (int64_t)(kInf - lc) : (int64_t)kInf;
                const int32_t minup = kInf - g.ctl->jminup_c[cur];
                int gg = l / g.Lg;
                while (gg + 1 < g.G && sh_upmax[gg + 1] < minup) ++gg;
                const int64_t top = (int64_t)(gg + 1) * g.Lg - 1;
                const int64_t x = lprev;
                const int64_t j = min(min(low - x - 3, other - x - 1), top - x - 1);
                if (j >= 1) {
                    skip = (int32_t)j;
                    if (T.leader()) {
                        const unsigned long long jm = (unsigned long long)j * (unsigned long long)mprev_n;
                        const unsigned long long jv = (unsigned long long)j * g.ctl->jsdeg[cur];
                        atomicAdd(&g.ctl->st[kStRounds], (unsigned long long)j);
                        atomicAdd(&g.ctl->st[kStMoves], jm);
                        atomicAdd(&g.ctl->st[kStVisits], jv);
                        atomicAdd(&g.ctl->st[kStSkipRounds], (unsigned long long)j);
                        atomicAdd(&g.ctl->st[kStSkipMoves], jm);
                        atomicAdd(&g.ctl->st[kStSkipVisits], jv);
                    }
                    l += skip;
                }
            }
        }
        lprev = l;
        if (l >= g.K - 1 || r > g.K + 4) {  // the top group is never violated
            if (T.leader()) report(g, kErrInternal, 21, l, r, 0);
            return false;
        }
        const int32_t flr = round_flag(r), flp = round_flag(r + 1);
        const int mi = r % 3, mprev = (r + 2) % 3;
        const uint64_t t_round = (g.trace && T.leader()) ? global_ns() : 0;
        // the list is rewritten (live entries only) once most of it has been taken
        const int32_t pc = g.ctl->jpend[pb], taken = g.ctl->jcons[pb];
        const bool compact = 2 * taken > pc || pc > g.n;
        const int pd = compact ? pb ^ 1 : pb;  // where this round's new entries go
        // phase A
        if (T.leader()) {
            g.ctl->jmov[(r + 1) % 3] = 0;  // last read in phase B of round r - 1
            g.ctl->jbig[nxt] = 0;
        }
        if (r > 0) {
            const int32_t pm = g.ctl->jmov[mprev];
            for (int i = T.tid(); i < pm; i += T.nthreads()) atomicAnd(&g.level[g.TL[mprev][i].x], ~flp);
        }
        int32_t cmin = kInf;  // lowest carried level
        for (int i0 = T.wid() * 32; i0 < pc; i0 += T.nwarps() * 32) {
            const int i = i0 + lane;
            const int4 e = i < pc ? g.P[pb][i] : make_int4(0, -1, 0, 0);
            const bool live = e.y >= 0;
            const bool mv = live && (e.y == l || (skip && e.y == l - skip));
            const bool carry = live && !mv;
            int32_t c = 0;
            if (mv) {
                if ((g.level[e.x] & kLevelMask) != e.y) report(g, kErrInternal, 22, e.x, g.level[e.x], e.y);
                if (e.y != l) atomicAdd(&g.level[e.x], l - e.y);  // the skipped rounds' moves
                atomicOr(&g.level[e.x], flr);
                c = g.cap[e.x];
                if (!compact) g.P[pb][i].y = -1;  // taken
            }
            if (!compact) {
                if (carry) cmin = min(cmin, e.y);  // never a mover of this round staying on
            } else {
                jump_push(g, pd, nxt, carry, e.x, e.y, true);
            }
            const bool big = mv && c > g.block_cap;
            const int pos = warp_append(&g.ctl->jmov[mi], mv);
            if (mv) g.TL[mi][pos] = make_int4(e.x, c, 0, 0);
            const int pbg = warp_append(&g.ctl->jbig[cur], big);
            if (big) g.M[0][pbg] = make_int4(e.x, c, 0, 0);
        }
        if (!compact) {  // the carried entries' lowest level, once per block
            cmin = (int32_t)__reduce_min_sync(kFull, (unsigned)cmin);
            if (lane == 0 && cmin < kInf) atomicMin(&bmin[0], cmin);
            __syncthreads();
            if (threadIdx.x == 0) {
                if (bmin[0] < kInf) {
                    atomicMax(&g.ctl->jnext_c[nxt], kInf - bmin[0]);
                    atomicMax(&g.ctl->jother_c[nxt], kInf - bmin[0]);
                }
                bmin[0] = kInf;
            }
        }
        if (!T.sync()) return false;
        const uint64_t t_a = (g.trace && T.leader()) ? global_ns() : 0;
        // the movers' targets: one warp per mover (a round's movers sit together in
        // the list, so the warps that found them would take them one after another),
        // a block per large table
        const int32_t mc = g.ctl->jmov[mi];
        const int32_t nb = g.ctl->jbig[cur];
        for (int i = T.wid(); i < mc; i += T.nwarps()) {
            const int4 it = g.TL[mi][i];
            if (it.y > g.block_cap) continue;
            const int32_t t = jump_target<false>(g, it.x, l, sh_upmax, whist, nullptr);
            if (lane == 0) g.dlv[it.x] = t;
        }
        for (int b = T.bid(); b < nb; b += T.nthreads() / blockDim.x) {
            const int32_t v = g.M[0][b].x;
            const int32_t t = jump_target<true>(g, v, l, sh_upmax, sh_block, sh_block + kWarpHist);
            if (threadIdx.x == 0) g.dlv[v] = t;
        }
        if (!T.sync()) return false;
        // phase B
        if (T.leader()) {
            atomicAdd(&g.ctl->st[kStRounds], 1ull);
            atomicAdd(&g.ctl->st[kStMoves], (unsigned long long)mc);
            // (every block read the list's counts at the start of the round, before phase A)
            if (compact) {  // the old list was read in phase A; it is the next compaction's target
                g.ctl->jpend[pb] = 0;
                g.ctl->jcons[pb] = 0;
            } else {
                g.ctl->jcons[pb] += mc;  // the entries taken in phase A are this round's movers
            }
            g.ctl->jnext_c[cur] = 0;  // read at the start of this round
            g.ctl->jstay[cur] = 0;
            g.ctl->jnonunit[cur] = 0;
            g.ctl->jother_c[cur] = 0;
            g.ctl->jlow_c[cur] = 0;
            g.ctl->jminup_c[cur] = 0;
            g.ctl->jsdeg[cur] = 0;
        }
        for (int i = T.wid(); i < mc; i += T.nwarps()) {
            const int4 it = g.TL[mi][i];
            if (it.y > g.block_cap) continue;
            const int32_t dg = jump_apply<false>(g, it.x, l, g.dlv[it.x], flr, pd, nxt, sh_upmax, nullptr, &aff);
            if (lane == 0) visits += dg;
        }
        for (int b = T.bid(); b < nb; b += T.nthreads() / blockDim.x) {
            const int32_t v = g.M[0][b].x;
            const int32_t dg = jump_apply<true>(g, v, l, g.dlv[v], flr, pd, nxt, sh_upmax, sh_block + kWarpHist, &aff);
            if (threadIdx.x == 0) visits += dg;
        }
        if (r > 0) {  // the previous round's movers that do not move now: target dropped
            const int32_t pm = g.ctl->jmov[mprev];
            for (int i = T.tid(); i < pm; i += T.nthreads()) {
                const int32_t v = g.TL[mprev][i].x;
                if (!(g.level[v] & flr)) g.dlv[v] = -1;
            }
        }
        if (!T.sync()) return false;
        if (g.trace && T.leader() && g.ctl->trace_n < g.trace_cap) {
            int32_t *rec = g.trace + 12 * g.ctl->trace_n++;
            rec[0] = l; rec[1] = 2; rec[2] = mc; rec[3] = nb; rec[4] = pc - taken;
            rec[5] = (int32_t)(global_ns() - t_round); rec[6] = (int32_t)(t_a - t_round); rec[7] = skip;
            rec[8] = g.ctl->jstay[nxt]; rec[9] = g.ctl->jnonunit[nxt];
            rec[10] = g.ctl->jother_c[nxt] ? kInf - g.ctl->jother_c[nxt] : -1;
            rec[11] = g.ctl->jlow_c[nxt] ? kInf - g.ctl->jlow_c[nxt] : -1;
        }
        pb = pd;
    }
    // the last round's movers lose their flag and their target (dlv back to -1)
    if (r > 0) {
        const int mlast = (r - 1) % 3;
        const int32_t pm = g.ctl->jmov[mlast];
        for (int i = T.tid(); i < pm; i += T.nthreads()) {
            const int32_t v = g.TL[mlast][i].x;
            atomicAnd(&g.level[v], kLevelMask);
            g.dlv[v] = -1;
        }
    }
    visits = warp_sum64(visits);
    const unsigned long long affs = warp_sum64(aff);
    if (lane == 0 && visits) atomicAdd(&g.ctl->st[kStVisits], visits);
    if (lane == 0 && affs) atomicAdd(&g.ctl->st[kStAffected], affs);
    if (!T.sync()) return false;
    return true;
}

// ---------------------------------------------------------------------------
// One whole batch (Algorithm 1, one half): returns early when the team stopped
// (error word set).  sh: shared memory with the group tables, a block-scan
// scratch and one histogram per warp (the first also serves block-wide
// desire-levels).
// ---------------------------------------------------------------------------
// Trace record 0: {kind, then the durations between consecutive marks}.
__device__ __forceinline__ void trace_steps(const GraphCtx &g, const uint64_t (&t)[8], int n, int32_t kind) {
    int32_t *rec = g.trace;
    rec[0] = kind;
    for (int i = 1; i < 12; ++i) rec[i] = (i < n) ? (int32_t)(t[i] - t[i - 1]) : 0;
}

// kRoundsOnly: the steps before the rounds already ran as separate kernels (the
// single-graph calls); they are compiled out, leaving the rounds kernel leaner.
template <class Team, bool kRoundsOnly = false>
__device__ void run_batch(Team &T, const GraphCtx &g, const BatchIn &in, int32_t *sh, int stage_shift) {
    int32_t *sh_upmax = sh;
    int32_t *sh_dnmin = sh + kMaxGroups;
    int *sh_scan = sh + 2 * kMaxGroups;  // 64 ints
    unsigned long long *sh_res = reinterpret_cast<unsigned long long *>(sh_scan);  // block_reserve: <= 17 slots
    int32_t *sh_block = sh + 2 * kMaxGroups + 64;  // kWarpHist + 32 ints, block-wide desire-levels
    int32_t *whist = sh_block + kWarpHist + 32 + (threadIdx.x >> 5) * kWarpHist;
    int32_t *sh_stage = sh_block + kWarpHist + 32 + (blockDim.x >> 5) * kWarpHist;
    for (int i = threadIdx.x; i < g.G; i += blockDim.x) {
        sh_upmax[i] = g.upmax[i];
        sh_dnmin[i] = g.dnmin[i];
    }
    if (g.test_delay_us > 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        const uint64_t t0 = global_ns();  // bounded: ends after test_delay_us
        while (global_ns() - t0 < (uint64_t)g.test_delay_us * 1000u) __nanosleep(1000);
    }
    __syncthreads();
    // diagnostics: record 0 of the trace holds the durations of the steps before the rounds
    const bool tr = g.trace && T.leader();
    uint64_t tmark[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int nmark = 0;
    if (tr) {
        g.ctl->trace_n = 1;
        tmark[nmark++] = global_ns();
    }
    if constexpr (kRoundsOnly) {  // a step kernel that failed stops the rounds too
        if (ld_volatile(&g.ctl->err)) return;
    } else if (in.B > 0) {
        pre_canon(T, g, in, sh_res);
        if (!T.sync()) return;  // ids outside [0,n): nothing has changed
        if (tr) tmark[nmark++] = global_ns();
        pre_filter(T, g, in, sh_res);
        if (!T.sync()) return;
        if (tr) tmark[nmark++] = global_ns();
    }
    if (in.op == kOpInsert) {
        if constexpr (!kRoundsOnly) {
            pre_grow_request(T, g, sh_res);
            if (!T.sync()) return;
            pre_pool_check(T, g);  // on a full pool: the incoming counts undone, kErrNeedPool
            if (!T.sync()) return;  // the host grows the pool and runs the batch again
            if (tr) tmark[nmark++] = global_ns();
            pre_alloc(T, g, sh_res);
            if (!T.sync()) return;
            pre_clear(T, g);
            if (!T.sync()) return;
            pre_grow(T, g);
            if (!T.sync()) return;
            pre_commit(T, g);
            if (!T.sync()) return;
            if (tr) tmark[nmark++] = global_ns();
            step_apply_insert(T, g);
            if (!T.sync()) return;
            if (tr) tmark[nmark++] = global_ns();
        }
        if (!g.jump && !ins_sort_candidates(T, g, sh_scan)) return;
        if (tr) {
            tmark[nmark++] = global_ns();
            trace_steps(g, tmark, nmark, -1);
        }
        if (g.jump) ins_rounds_jump(T, g, sh_upmax, whist, sh_block);
        else ins_rounds(T, g, sh_upmax, whist, stage_setup(sh_stage, stage_shift));
    } else {
        if constexpr (!kRoundsOnly) {
            if (T.leader()) {
                g.ctl->nextmin[0] = kInf;
                g.ctl->nextmin[1] = kInf;
            }
            step_apply_delete(T, g);
            if (!T.sync()) return;
            if (tr) tmark[nmark++] = global_ns();
            pre_shrink_plan(T, g, sh_res);
            if (!T.sync()) return;
            pre_shrink_a(T, g);
            if (!T.sync()) return;
            pre_shrink_b(T, g);
            if (!T.sync()) return;
            pre_shrink_c(T, g);
            if (!T.sync()) return;
            if (tr) tmark[nmark++] = global_ns();
        }
        unsigned long long evals = 0, evisits = 0;
        if (!dl_batch(T, g, g.touched, g.ctl->tcount, 0, -1, sh_dnmin, whist, sh_block, evals, evisits)) return;
        if (evals) {
            atomicAdd(&g.ctl->st[kStDlEvals], evals);
            atomicAdd(&g.ctl->st[kStDlVisits], evisits);
        }
        if (!T.sync()) return;
        if (tr) {
            tmark[nmark++] = global_ns();
            trace_steps(g, tmark, nmark, -2);
            g.trace[8] = g.ctl->tcount;   // vertices the batch touched
            g.trace[9] = g.ctl->rcnt[1];  // of them violating, desire-level by a warp
            g.trace[10] = g.ctl->rbcnt;   // by a block (tables above block_cap)
        }
        if (T.leader()) {
            g.ctl->rcnt[1] = 0;
            g.ctl->rbcnt = 0;
        }
        del_rounds(T, g, in.stamp_base, sh_dnmin, whist, sh_block, whist, stage_setup(sh_stage, stage_shift));
    }
}

}  // namespace pl
