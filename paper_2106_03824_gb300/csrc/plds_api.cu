// Host runtime and C ABI of the GB300 PLDS (declared in include/plds.h).
//
// One batch call = the steps before the level rounds (preprocessing, table
// growth or shrinking, adjacency and counter updates) as plain full-occupancy
// kernels, then one cooperative kernel for the level rounds with grid-wide
// barriers between rounds, followed by one read of the control words.  The
// serving and batched forms run the same device steps inside their persistent
// kernels with team barriers between them.  Device memory comes from the caller's allocator (default:
// cudaMallocAsync on the handle's stream).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>
#include <new>
#include <time.h>
#include <vector>

#include "plds.h"
#include "plds_device.cuh"
#include "plds_tables.h"

using namespace pl;

static thread_local int g_last_status = PLDS_OK;

static int set_status(int s) {
    g_last_status = s;
    return s;
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
// The level rounds of one batch (after the step kernels below), one cooperative
// launch: 152 blocks (one per SM) x 512 threads, grid barriers between rounds.
__global__ void __launch_bounds__(512) k_batch_grid(const __grid_constant__ GraphCtx g) {
    extern __shared__ int32_t sh[];
    GridTeam T{g.ctl, g.wait_limit_ns, g.barrier_sleep_ns};
    run_batch<GridTeam, true>(T, g, BatchIn{g.edges, g.B, g.op, g.stamp_base}, sh, 0);
}

// The steps before the level rounds (preprocessing, table growth and shrinking,
// adjacency and counter updates) as plain kernels for the single-graph batch
// calls: they need no grid barrier -- each kernel boundary orders one step against
// the next -- so they run at full occupancy instead of one block per SM.  Each
// starts by reading the error word: a step that failed (bad id, pool too small)
// stops the rest, and the cooperative rounds kernel after them as well.
constexpr int kPreThreads = 256;
#define PRE_SCRATCH             \
    FreeTeam T;                 \
    __shared__ unsigned long long sh_res[kPreThreads / 32 + 1]

__global__ void __launch_bounds__(kPreThreads) k_pre_canon_filter(const __grid_constant__ GraphCtx g) {
    PRE_SCRATCH;
    pre_canon_filter(T, g, BatchIn{g.edges, g.B, g.op, g.stamp_base}, sh_res);
}

// After an insertion batch was rejected for an id outside [0, n): the incoming
// counts of the touched vertices back to zero (they are per batch).
__global__ void k_undo_inc(const int32_t *__restrict__ touched, int64_t count, int32_t *inc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        inc[touched[i]] = 0;
}

__global__ void __launch_bounds__(kPreThreads) k_pre_grow_request(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    PRE_SCRATCH;
    pre_grow_request(T, g, sh_res);
}

__global__ void __launch_bounds__(kPreThreads) k_pre_pool_check(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    FreeTeam T;
    pre_pool_check(T, g);
}

__global__ void __launch_bounds__(kPreThreads) k_pre_alloc(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    PRE_SCRATCH;
    pre_alloc(T, g, sh_res);
}

__global__ void __launch_bounds__(kPreThreads) k_pre_clear(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    FreeTeam T;
    pre_clear(T, g);
}

__global__ void __launch_bounds__(kPreThreads) k_pre_grow(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    FreeTeam T;
    pre_grow(T, g);
}

__global__ void __launch_bounds__(kPreThreads) k_pre_commit(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    FreeTeam T;
    pre_commit(T, g);
}

__global__ void __launch_bounds__(kPreThreads) k_pre_apply_insert(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    FreeTeam T;
    step_apply_insert(T, g);
}

__global__ void __launch_bounds__(kPreThreads) k_pre_apply_delete(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    FreeTeam T;
    if (T.leader()) {
        g.ctl->nextmin[0] = kInf;
        g.ctl->nextmin[1] = kInf;
    }
    step_apply_delete(T, g);
}

__global__ void __launch_bounds__(kPreThreads) k_pre_shrink_plan(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    PRE_SCRATCH;
    pre_shrink_plan(T, g, sh_res);
}

__global__ void __launch_bounds__(kPreThreads) k_pre_shrink_a(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    FreeTeam T;
    pre_shrink_a(T, g);
}

__global__ void __launch_bounds__(kPreThreads) k_pre_shrink_b(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    FreeTeam T;
    pre_shrink_b(T, g);
}

__global__ void __launch_bounds__(kPreThreads) k_pre_shrink_c(const __grid_constant__ GraphCtx g) {
    if (ld_volatile(&g.ctl->err)) return;
    FreeTeam T;
    pre_shrink_c(T, g);
}

// Coreness estimate (Definition "Coreness Estimate"): exponent
// max(floor((level+1)/Lg) - 1, 0), or -1 (estimate 0) for degree 0.
__global__ void k_coreness(const int32_t *__restrict__ level, const int32_t *__restrict__ deg, int32_t n,
                           int32_t Lg, const double *__restrict__ powtab, double *out_est, int32_t *out_exp) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t g = -1;
        if (deg[v] > 0) g = max((level[v] + 1) / Lg - 1, 0);
        if (out_est) out_est[v] = g < 0 ? 0.0 : powtab[g];
        if (out_exp) out_exp[v] = g;
    }
}

// Pool compaction: new offsets = exclusive prefix sum of table sizes.
__global__ void k_scan_block_sums(const int32_t *__restrict__ cap, int32_t n, long long *bsum) {
    __shared__ long long s[32];
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    long long x = v < n ? cap[v] : 0;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s[i];
        bsum[blockIdx.x] = t;
    }
}

__global__ void k_scan_top(long long *bsum, int32_t nb, long long *total) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        long long run = 0;
        for (int i = 0; i < nb; ++i) {
            long long t = bsum[i];
            bsum[i] = run;
            run += t;
        }
        *total = run;
    }
}

__global__ void k_scan_apply(const int32_t *__restrict__ cap, int32_t n, const long long *bsum, int64_t *newoff) {
    __shared__ long long s[33];
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    long long x = v < n ? cap[v] : 0, incl = x;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s[w] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            long long t = s[i];
            s[i] = run;
            run += t;
        }
    }
    __syncthreads();
    if (v < n) newoff[v] = bsum[blockIdx.x] + s[w] + incl - x;
}

__global__ void k_pool_copy(const int32_t *__restrict__ oldp, int32_t *__restrict__ newp, int64_t *off,
                            const int64_t *__restrict__ newoff, const int32_t *__restrict__ cap, int32_t n) {
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int lane = threadIdx.x & 31;
    for (int64_t v = warp; v < n; v += nw) {
        int32_t c = cap[v];
        const int4 *src = reinterpret_cast<const int4 *>(oldp + off[v]);
        int4 *dst = reinterpret_cast<int4 *>(newp + newoff[v]);
        for (int j = lane; j < (c >> 2); j += 32) dst[j] = src[j];
        __syncwarp();
        if (lane == 0) off[v] = newoff[v];
    }
}

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct plds {
    int device = 0;
    cudaStream_t stream = nullptr;
    plds_allocator alloc{};
    bool custom_alloc = false;
    bool poisoned = false;
    int32_t n = 0;
    bool jump = false;  // insertion: the jump variant (PLDS_FLAG_JUMP)
    // what plds_create_ex was given (plds_autotune builds scratch handles alike)
    double delta = 0, lambda = 0;
    int32_t levels_per_group = 0;
    uint32_t flags = 0;
    Tables T;
    plds_tuning tune{};
    int64_t wait_limit_ns = 20ll * 1000 * 1000 * 1000;
    int num_sms = 0;
    int32_t stamp_base = 1;
    int64_t device_bytes = 0;
    int64_t pool_grows = 0;
    plds_stats_t last{};
    int64_t launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evm = nullptr;  // batch start, end; end of the step kernels
    // persistent state
    DevBuf upmax, dnmin, powtab, level, deg, up, upstar, off, cap, tomb, stamp, dlv, dslack, inc;
    DevBuf pool, pool_top, ctl;
    int64_t pool_cap = 0;
    int64_t pool_live = 0;   // slots in use after the last compaction
    // orientation tracking: levels before the last batch call, its kind, validity
    DevBuf old_level, oscratch, okeys;
    DevBuf sk_scratch, sk_tables, sk_ctl;  // static approximate k-core
    int32_t orient_op = -1;
    bool orient_ok = false;
    int64_t pool_limit = 0;  // bytes a grown pool may take (0: free HBM only)
    // scratch: n-sized
    DevBuf acc, M[2], TL[3], P[2], R, R2, bins, levlist, CL[3];
    DevBuf lbuf[3], lout, lfill[2];  // insertion up-lists
    int64_t clcap = 0, lcap = 0;
    // scratch: batch-sized
    DevBuf edges, hset, ukeys, vkeys, touched, S, arena, trace;
    int64_t bcap = 0, hcap = 0, tcap = 0, arena_cap = 0;
    Ctl host_ctl{};
};

static void *dev_alloc(plds *h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (h->custom_alloc) {
        p = h->alloc.alloc(bytes, (void *)h->stream, h->alloc.ctx);
    } else if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

static void dev_free(plds *h, DevBuf &b) {
    if (!b.p) return;
    if (h->custom_alloc) h->alloc.free(b.p, b.bytes, (void *)h->stream, h->alloc.ctx);
    else cudaFreeAsync(b.p, h->stream);
    h->device_bytes -= (int64_t)b.bytes;
    b.p = nullptr;
    b.bytes = 0;
}

static bool dev_get(plds *h, DevBuf &b, size_t bytes) {
    if (b.p && b.bytes >= bytes) return true;
    dev_free(h, b);
    b.p = dev_alloc(h, bytes);
    if (!b.p) return false;
    b.bytes = bytes ? bytes : 16;
    h->device_bytes += (int64_t)b.bytes;
    return true;
}

template <class T>
static T *P(DevBuf &b) {
    return reinterpret_cast<T *>(b.p);
}

static int cuda_check(plds *h) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        h->poisoned = true;
        return PLDS_EDEVICE;
    }
    return PLDS_OK;
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int64_t pow2_at_least(int64_t x) {
    int64_t c = 1;
    while (c < x) c <<= 1;
    return c;
}

static void free_all(plds *h) {
    DevBuf *bufs[] = {&h->upmax, &h->dnmin, &h->powtab, &h->level, &h->deg,   &h->up,    &h->upstar,
                      &h->off,   &h->cap,   &h->tomb,   &h->stamp, &h->dlv,   &h->dslack, &h->inc,   &h->pool,
                      &h->pool_top, &h->ctl, &h->acc,   &h->M[0],  &h->M[1],  &h->TL[0], &h->TL[1], &h->TL[2],
                      &h->P[0],  &h->P[1],  &h->R, &h->R2,     &h->bins,  &h->levlist, &h->CL[0], &h->CL[1],
                      &h->CL[2], &h->edges, &h->hset,   &h->ukeys, &h->vkeys, &h->touched, &h->S, &h->arena, &h->trace,
                      &h->old_level, &h->oscratch, &h->okeys, &h->sk_scratch, &h->sk_tables, &h->sk_ctl,
                      &h->lbuf[0], &h->lbuf[1], &h->lbuf[2], &h->lout, &h->lfill[0], &h->lfill[1]};
    for (DevBuf *b : bufs) dev_free(h, *b);
}

// Chunk-item lists (one 128-slot chunk of every table, plus one item per vertex) and
// the insertion up-list buffers (as many entries as the pool, at most 2^27 each: a
// mover whose list does not fit is scanned from its table again).
static bool alloc_chunk_lists(plds *h) {
    int64_t need = h->pool_cap / kChunk + (int64_t)h->n + 1024;
    if (h->clcap < need) {
        for (int i = 0; i < 3; ++i)
            if (!dev_get(h, h->CL[i], sizeof(int4) * (size_t)need)) return false;
        h->clcap = need;
    }
    const int64_t lneed = (std::min<int64_t>(std::max<int64_t>(h->pool_cap, 4096), (int64_t)1 << 27) + 3) & ~(int64_t)3;
    if (h->lcap < lneed) {
        for (int i = 0; i < 3; ++i)
            if (!dev_get(h, h->lbuf[i], sizeof(int32_t) * (size_t)lneed)) return false;
        h->lcap = lneed;
    }
    return true;
}

static bool ensure_batch_scratch(plds *h, int64_t B) {
    if (B <= h->bcap) return true;
    int64_t bc = std::max<int64_t>(B, 1024);
    int64_t hc = pow2_at_least(2 * bc);
    int64_t tc = std::min<int64_t>(2 * bc, (int64_t)h->n);
    int64_t ac = std::max<int64_t>(2 * bc, 1 << 20);
    if (!dev_get(h, h->edges, sizeof(int2) * (size_t)bc) || !dev_get(h, h->hset, 8 * (size_t)hc) ||
        !dev_get(h, h->ukeys, 8 * (size_t)bc) || !dev_get(h, h->vkeys, 8 * (size_t)bc) ||
        !dev_get(h, h->touched, 4 * (size_t)tc) || !dev_get(h, h->S, 4 * (size_t)tc) ||
        !dev_get(h, h->arena, 4 * (size_t)ac))
        return false;
    h->bcap = bc;
    h->hcap = hc;
    h->tcap = tc;
    h->arena_cap = ac;
    return true;
}

static int block_threads(const plds *h) { return h->tune.block_threads > 0 ? h->tune.block_threads : 512; }

// Dynamic shared memory of a batch kernel block: group tables, scan scratch,
// block-wide desire-level histogram, one histogram per warp, staging area.
static size_t smem_bytes(int threads, int stage_shift = 0) {
    return sizeof(int32_t) *
           (size_t)(2 * kMaxGroups + 64 + kWarpHist + 32 + (threads / 32) * kWarpHist + stage_ints(stage_shift));
}

// Device memory that pool growth and serving admission leave free for everything else.
constexpr int64_t kHbmReserve = 1ll << 30;

// Move every table into a new pool laid out back to back, with room for `extra`
// more slots; the old pool is freed.
static int grow_pool(plds *h, int64_t extra) {
    const int threads = 1024;
    int32_t nb = (int32_t)((h->n + threads - 1) / threads);
    DevBuf bsum, newoff, total;
    if (!dev_get(h, bsum, sizeof(long long) * (size_t)(nb + 1)) || !dev_get(h, newoff, 8 * (size_t)h->n) ||
        !dev_get(h, total, 8)) {
        dev_free(h, bsum);
        dev_free(h, newoff);
        dev_free(h, total);
        return PLDS_ENOMEM;
    }
    h->launches += 4;
    k_scan_block_sums<<<nb, threads, 0, h->stream>>>(P<int32_t>(h->cap), h->n, P<long long>(bsum));
    k_scan_top<<<1, 32, 0, h->stream>>>(P<long long>(bsum), nb, P<long long>(total));
    k_scan_apply<<<nb, threads, 0, h->stream>>>(P<int32_t>(h->cap), h->n, P<long long>(bsum), P<int64_t>(newoff));
    long long live = 0;
    cudaMemcpyAsync(&live, total.p, 8, cudaMemcpyDeviceToHost, h->stream);
    cudaStreamSynchronize(h->stream);
    int rc = cuda_check(h);
    if (rc) return rc;
    // four times the live slots: every growth costs a stopped attempt, a copy of the
    // pool and a rerun, so fewer of them pay for the extra room (capped by free HBM)
    int64_t want = std::max<int64_t>(h->pool_cap, 4 * (live + extra));
    want = (want + 3) & ~(int64_t)3;
    // gate on free HBM (keep kHbmReserve free for everything else on the device)
    // and on the pool limit, if one is set
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        free_b = 0;
    }
    int64_t avail = (int64_t)free_b - kHbmReserve;
    if (h->pool_limit > 0) avail = std::min<int64_t>(avail, h->pool_limit);
    if (avail < 4 * want) {
        const int64_t fit = avail / 4;
        want = std::max<int64_t>(live + extra + 4, fit) & ~(int64_t)3;
        if (want < live + extra) {
            dev_free(h, bsum);
            dev_free(h, newoff);
            dev_free(h, total);
            return PLDS_ENOMEM;
        }
    }
    cudaGetLastError();
    if (want / 4 >= ((int64_t)1 << 31)) {  // scan items address the pool in int32 units of 4 slots
        dev_free(h, bsum);
        dev_free(h, newoff);
        dev_free(h, total);
        return PLDS_ENOMEM;
    }
    DevBuf np;
    if (!dev_get(h, np, 4 * (size_t)want)) {
        dev_free(h, bsum);
        dev_free(h, newoff);
        dev_free(h, total);
        return PLDS_ENOMEM;
    }
    k_pool_copy<<<std::max(1, h->num_sms * 8), 256, 0, h->stream>>>(P<int32_t>(h->pool), P<int32_t>(np),
                                                                     P<int64_t>(h->off), P<int64_t>(newoff),
                                                                     P<int32_t>(h->cap), h->n);
    unsigned long long top = (unsigned long long)live;
    cudaMemcpyAsync(h->pool_top.p, &top, 8, cudaMemcpyHostToDevice, h->stream);
    cudaStreamSynchronize(h->stream);
    dev_free(h, h->pool);
    h->pool = np;
    h->pool_cap = want;
    h->pool_live = live;
    h->pool_grows++;
    dev_free(h, bsum);
    dev_free(h, newoff);
    dev_free(h, total);
    if (!alloc_chunk_lists(h)) return PLDS_ENOMEM;
    return cuda_check(h);
}

// Default thread cutoff of a batch (tuning field 0).  Measured on R-MAT scale 20
// (Ins and Del protocols): 8 slots save 2-4 % on deletion batches and on insertion
// batches of 10^5 edges, 16 slots save 3 % on insertion batches of 10^6.  The
// serving loop's context (B = 0: batches of every size) keeps 16.
static int32_t default_thread_cap(int32_t op, int64_t B) {
    if (B <= 0) return 16;
    return (op == kOpDelete || B <= 300000) ? 8 : 16;
}

static GraphCtx make_ctx(plds *h, int32_t op, const int32_t *edges, int64_t B) {
    GraphCtx g{};
    g.n = h->n;
    g.Lg = h->T.Lg;
    g.K = h->T.K;
    g.G = h->T.G;
    g.op = op;
    g.stamp_base = h->stamp_base;
    g.thread_max_cap = h->tune.thread_max_cap > 0 ? h->tune.thread_max_cap : default_thread_cap(op, B);
    g.load_num = h->tune.load_num > 0 ? h->tune.load_num : 3;
    g.load_den = h->tune.load_den > 0 ? h->tune.load_den : 4;
    g.block_cap = h->tune.block_cap > 0 ? h->tune.block_cap : 1024;
    g.list_cap = h->tune.list_cap > 0 ? h->tune.list_cap : 256;
    g.jump = h->jump ? 1 : 0;
    g.wait_limit_ns = h->wait_limit_ns;
    g.test_delay_us = h->tune.test_delay_us;
    g.barrier_sleep_ns = h->tune.barrier_sleep_ns == 0 ? 32 : (h->tune.barrier_sleep_ns < 0 ? 0 : h->tune.barrier_sleep_ns);
    g.upmax = P<int32_t>(h->upmax);
    g.dnmin = P<int32_t>(h->dnmin);
    g.level = P<int32_t>(h->level);
    g.deg = P<int32_t>(h->deg);
    g.up = P<int32_t>(h->up);
    g.upstar = P<int32_t>(h->upstar);
    g.off = P<int64_t>(h->off);
    g.cap = P<int32_t>(h->cap);
    g.tomb = P<int32_t>(h->tomb);
    g.stamp = P<int32_t>(h->stamp);
    g.dlv = P<int32_t>(h->dlv);
    g.dslack = P<int32_t>(h->dslack);
    g.inc = P<int32_t>(h->inc);
    g.slots = P<int32_t>(h->pool);
    g.pool_top = P<unsigned long long>(h->pool_top);
    g.pool_cap = h->pool_cap;
    g.edges = edges;
    g.B = B;
    g.hset = P<unsigned long long>(h->hset);
    g.hcap = h->hcap;
    g.ukeys = P<unsigned long long>(h->ukeys);
    g.vkeys = P<unsigned long long>(h->vkeys);
    g.touched = P<int32_t>(h->touched);
    g.S = P<int32_t>(h->S);
    g.bins = P<int32_t>(h->bins);
    g.levlist = P<int32_t>(h->levlist);
    for (int i = 0; i < 2; ++i) {
        g.M[i] = P<int4>(h->M[i]);
        g.P[i] = P<int4>(h->P[i]);
    }
    for (int i = 0; i < 3; ++i) {
        g.TL[i] = P<int4>(h->TL[i]);
        g.CL[i] = P<int4>(h->CL[i]);
    }
    g.acc = P<unsigned long long>(h->acc);
    for (int i = 0; i < 3; ++i) g.lbuf[i] = P<int32_t>(h->lbuf[i]);
    g.lcap = h->lcap;
    g.lout = P<int32_t>(h->lout);
    g.lfill[0] = P<int32_t>(h->lfill[0]);
    g.lfill[1] = P<int32_t>(h->lfill[1]);
    g.R[0] = P<int32_t>(h->R);
    g.R[1] = P<int32_t>(h->R2);
    g.clcap = h->clcap;
    g.arena = P<int32_t>(h->arena);
    g.arena_cap = h->arena_cap;
    g.trace = h->tune.trace_rounds ? P<int32_t>(h->trace) : nullptr;
    g.trace_cap = h->tune.trace_rounds ? (int32_t)(h->trace.bytes / 48) : 0;
    g.ctl = P<Ctl>(h->ctl);
    return g;
}

// A kernel's dynamic shared-memory limit is an attribute of the kernel on one
// device: raise it once per device (any host thread may drive handles on any
// device), the first time a kernel launches there.
constexpr int kAttrDevices = 128;

template <class K>
static void raise_smem_limit(K kernel, std::atomic<bool> (&done)[kAttrDevices], int device) {
    if (device >= 0 && device < kAttrDevices && done[device].load(std::memory_order_acquire)) return;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (device >= 0 && device < kAttrDevices) done[device].store(true, std::memory_order_release);
}

static std::atomic<bool> g_attr_batch[kAttrDevices];

// The step kernels of one batch attempt, in stream order, then pre_done set so
// that the cooperative kernel starts at the rounds.  Records ev0 before them and
// evm after them.
static void launch_pre(plds *h, GraphCtx &g) {
    const int blocks = std::max(1, h->num_sms * 8);
    cudaStream_t s = h->stream;
    cudaEventRecord(h->ev0, s);
    int k = 0;
    if (g.B > 0) {
        k_pre_canon_filter<<<blocks, kPreThreads, 0, s>>>(g);
        k += 1;
    }
    if (g.op == kOpInsert) {
        k_pre_grow_request<<<blocks, kPreThreads, 0, s>>>(g);
        k_pre_pool_check<<<blocks, kPreThreads, 0, s>>>(g);
        k_pre_alloc<<<blocks, kPreThreads, 0, s>>>(g);
        k_pre_clear<<<blocks, kPreThreads, 0, s>>>(g);
        k_pre_grow<<<blocks, kPreThreads, 0, s>>>(g);
        k_pre_commit<<<blocks, kPreThreads, 0, s>>>(g);
        k_pre_apply_insert<<<blocks, kPreThreads, 0, s>>>(g);
        k += 7;
    } else {
        k_pre_apply_delete<<<blocks, kPreThreads, 0, s>>>(g);
        k_pre_shrink_plan<<<blocks, kPreThreads, 0, s>>>(g);
        k_pre_shrink_a<<<blocks, kPreThreads, 0, s>>>(g);
        k_pre_shrink_b<<<blocks, kPreThreads, 0, s>>>(g);
        k_pre_shrink_c<<<blocks, kPreThreads, 0, s>>>(g);
        k += 5;
    }
    cudaEventRecord(h->evm, s);
    h->launches += k;
    g.pre_done = 1;
}

// An insertion batch rejected for an id outside [0, n) by the one-pass step
// kernel: its valid keys' incoming counts are cleared, leaving the graph as before.
static void undo_incoming(plds *h, const Ctl &c, const GraphCtx &g) {
    if (g.op != kOpInsert || c.ttotal == 0) return;
    const int64_t cnt = (int64_t)c.ttotal;
    const int blocks = (int)std::min<int64_t>((cnt + 255) / 256, (int64_t)h->num_sms * 8);
    k_undo_inc<<<blocks, 256, 0, h->stream>>>(g.touched, cnt, g.inc);
    h->launches++;
    cudaStreamSynchronize(h->stream);
}

static int launch_batch(plds *h, const GraphCtx &g) {
    const int threads = block_threads(h);
    const size_t smem = smem_bytes(threads);
    raise_smem_limit(k_batch_grid, g_attr_batch, h->device);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_grid, threads, smem);
    int per_sm = h->tune.blocks_per_sm > 0 ? std::min(h->tune.blocks_per_sm, occ) : 1;
    if (per_sm < 1) return PLDS_EDEVICE;
    dim3 grid(h->num_sms * per_sm), block(threads);
    void *args[] = {(void *)&g};
    if (!g.pre_done) cudaEventRecord(h->ev0, h->stream);
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_batch_grid, grid, block, args, smem, h->stream);
    cudaEventRecord(h->ev1, h->stream);
    h->launches++;
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->poisoned = true;
        return PLDS_EDEVICE;
    }
    return PLDS_OK;
}

static int run_op(plds *h, const int32_t *edges, int64_t B, int32_t op) {
    if (!h) return PLDS_EINVAL;
    if (h->poisoned) return PLDS_EPOISONED;
    if (B < 0 || (B > 0 && !edges)) return PLDS_EINVAL;
    std::memset(&h->last, 0, sizeof(h->last));
    h->last.submitted = B;
    h->orient_ok = false;
    cudaSetDevice(h->device);
    if (h->tune.track_orientation) {  // levels before the batch, for plds_flips / plds_oriented_updates
        if (!dev_get(h, h->old_level, 4 * (size_t)h->n)) return PLDS_ENOMEM;
        cudaMemcpyAsync(h->old_level.p, h->level.p, 4 * (size_t)h->n, cudaMemcpyDeviceToDevice, h->stream);
        h->host_ctl.vcount = 0;
        h->orient_op = op;
        if (B == 0) {
            h->orient_ok = true;
            return PLDS_OK;
        }
    }
    if (B == 0) return PLDS_OK;
    if (!ensure_batch_scratch(h, B)) return PLDS_ENOMEM;
    const int32_t *dedges = edges;
    if (!is_device_ptr(edges)) {
        cudaMemcpyAsync(h->edges.p, edges, sizeof(int32_t) * 2 * (size_t)B, cudaMemcpyHostToDevice, h->stream);
        dedges = P<int32_t>(h->edges);
    }
    for (int attempt = 0; attempt < 4; ++attempt) {
        if ((int64_t)h->stamp_base + 2 * (int64_t)h->T.K + 8 >= 0x7fffffff) {
            cudaMemsetAsync(h->stamp.p, 0, sizeof(int32_t) * (size_t)h->n, h->stream);
            h->stamp_base = 1;
        }
        cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), h->stream);
        cudaMemsetAsync(h->hset.p, 0xff, 8 * (size_t)h->hcap, h->stream);
        if (op == kOpInsert) cudaMemsetAsync(h->bins.p, 0, sizeof(int32_t) * ((size_t)h->T.K + 1), h->stream);
        GraphCtx g = make_ctx(h, op, dedges, B);
        h->stamp_base += h->T.K + 2;
        launch_pre(h, g);
        int rc = launch_batch(h, g);
        if (rc) return rc;
        cudaMemcpyAsync(&h->host_ctl, h->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
            cudaGetLastError();
            h->poisoned = true;
            return PLDS_EDEVICE;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) h->last.kernel_ns += (int64_t)(ms * 1e6);
        if (cudaEventElapsedTime(&ms, h->ev0, h->evm) == cudaSuccess) h->last.pre_ns += (int64_t)(ms * 1e6);
        cudaGetLastError();
        const Ctl &c = h->host_ctl;
        h->last.err_bits = c.err;
        h->last.err_site = c.err_site;
        h->last.err_info[0] = c.err_info[0];
        h->last.err_info[1] = c.err_info[1];
        h->last.err_info[2] = c.err_info[2];
        if (c.err == 0) break;
        if (c.err & kErrTimeout) {
            h->poisoned = true;
            return PLDS_ETIMEOUT;
        }
        if (c.err & kErrInvalidId) {
            undo_incoming(h, c, g);
            return PLDS_EINVAL;
        }
        if (c.err == kErrNeedPool && attempt < 3) {
            rc = grow_pool(h, (int64_t)c.grow_total);
            if (rc) return rc;
            continue;
        }
        h->poisoned = true;
        return PLDS_EINTERNAL;
    }
    const Ctl &c = h->host_ctl;
    h->last.err_bits = c.err;
    h->last.err_site = c.err_site;
    h->last.err_info[0] = c.err_info[0];
    h->last.err_info[1] = c.err_info[1];
    h->last.err_info[2] = c.err_info[2];
    h->last.self_loops = (int64_t)c.st[kStSelfLoops];
    h->last.duplicates = B - h->last.self_loops - (int64_t)c.ucount;
    h->last.filtered = (int64_t)c.st[kStFiltered];
    h->last.valid = (int64_t)c.vcount;
    h->last.rounds = (int64_t)c.st[kStRounds];
    h->last.moves = (int64_t)c.st[kStMoves];
    h->last.visits = (int64_t)c.st[kStVisits];
    h->last.dl_evals = (int64_t)c.st[kStDlEvals];
    h->last.dl_visits = (int64_t)c.st[kStDlVisits];
    h->last.slots_scanned = (int64_t)c.st[kStSlotsScanned];
    h->last.up_visits = (int64_t)c.st[kStUpVisits];
    h->last.affected = (int64_t)c.st[kStAffected];
    h->last.skipped_rounds = (int64_t)c.st[kStSkipRounds];
    h->last.skipped_moves = (int64_t)c.st[kStSkipMoves];
    h->last.skipped_visits = (int64_t)c.st[kStSkipVisits];
    h->last.skipped_up_visits = (int64_t)c.st[kStSkipUpVisits];
    h->orient_ok = h->tune.track_orientation != 0;
    return PLDS_OK;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

plds_t *plds_create_ex(int32_t n, double delta, double lambda, int32_t levels_per_group,
                       const plds_allocator *allocator, void *stream, uint32_t flags) {
    if ((flags & ~(uint32_t)(PLDS_FLAG_HEURISTIC | PLDS_FLAG_JUMP)) != 0 ||
        (allocator && (!allocator->alloc || !allocator->free))) {
        set_status(PLDS_EINVAL);
        return nullptr;
    }
    plds *h = new (std::nothrow) plds();
    if (!h) {
        set_status(PLDS_ENOMEM);
        return nullptr;
    }
    if (build_tables(n, delta, lambda, levels_per_group, &h->T, (flags & PLDS_FLAG_HEURISTIC) != 0) != 0) {
        delete h;
        set_status(PLDS_EINVAL);
        return nullptr;
    }
    cudaGetDevice(&h->device);
    if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
        cudaEventCreate(&h->evm) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        set_status(PLDS_EDEVICE);
        return nullptr;
    }
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    h->stream = (cudaStream_t)stream;
    if (allocator) {
        h->alloc = *allocator;
        h->custom_alloc = true;
    }
    h->n = n;
    h->jump = (flags & PLDS_FLAG_JUMP) != 0;
    h->delta = delta;
    h->lambda = lambda;
    h->levels_per_group = levels_per_group;
    h->flags = flags;
    const size_t N = (size_t)n;
    const size_t G = (size_t)h->T.G, K = (size_t)h->T.K;
    h->pool_cap = std::max<int64_t>(1 << 20, 8 * (int64_t)n);
    bool ok = dev_get(h, h->upmax, 4 * G) && dev_get(h, h->dnmin, 4 * G) && dev_get(h, h->powtab, 8 * G) &&
              dev_get(h, h->level, 4 * N) && dev_get(h, h->deg, 4 * N) && dev_get(h, h->up, 4 * N) &&
              dev_get(h, h->upstar, 4 * N) && dev_get(h, h->off, 8 * N) && dev_get(h, h->cap, 4 * N) &&
              dev_get(h, h->tomb, 4 * N) && dev_get(h, h->stamp, 4 * N) && dev_get(h, h->dlv, 4 * N) &&
              dev_get(h, h->dslack, 4 * N) &&
              dev_get(h, h->inc, 4 * N) && dev_get(h, h->pool, 4 * (size_t)h->pool_cap) &&
              dev_get(h, h->pool_top, 8) && dev_get(h, h->ctl, sizeof(Ctl)) && dev_get(h, h->acc, 8 * N) &&
              dev_get(h, h->lout, 4 * N) && dev_get(h, h->lfill[0], 4 * N) && dev_get(h, h->lfill[1], 4 * N) &&
              dev_get(h, h->M[0], 16 * N) && dev_get(h, h->M[1], 16 * N) && dev_get(h, h->TL[0], 16 * N) &&
              dev_get(h, h->TL[1], 16 * N) && dev_get(h, h->TL[2], 16 * N) && dev_get(h, h->P[0], 32 * N) &&
              dev_get(h, h->P[1], 32 * N) && dev_get(h, h->R, 4 * N) && dev_get(h, h->R2, 4 * N) && dev_get(h, h->bins, 4 * (K + 1)) &&
              dev_get(h, h->levlist, 4 * (K + 1)) && alloc_chunk_lists(h);
    if (!ok) {
        free_all(h);
        cudaStreamSynchronize(h->stream);
        delete h;
        set_status(PLDS_ENOMEM);
        return nullptr;
    }
    cudaStream_t s = h->stream;
    cudaMemcpyAsync(h->upmax.p, h->T.upmax.data(), 4 * G, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->dnmin.p, h->T.dnmin.data(), 4 * G, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(h->powtab.p, h->T.pow.data(), 8 * G, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(h->level.p, 0, 4 * N, s);
    cudaMemsetAsync(h->deg.p, 0, 4 * N, s);
    cudaMemsetAsync(h->up.p, 0, 4 * N, s);
    cudaMemsetAsync(h->upstar.p, 0, 4 * N, s);
    cudaMemsetAsync(h->off.p, 0, 8 * N, s);
    cudaMemsetAsync(h->cap.p, 0, 4 * N, s);
    cudaMemsetAsync(h->tomb.p, 0, 4 * N, s);
    cudaMemsetAsync(h->stamp.p, 0, 4 * N, s);
    cudaMemsetAsync(h->dlv.p, 0xff, 4 * N, s);
    cudaMemsetAsync(h->inc.p, 0, 4 * N, s);
    cudaMemsetAsync(h->acc.p, 0, 8 * N, s);
    cudaMemsetAsync(h->pool_top.p, 0, 8, s);
    cudaStreamSynchronize(s);
    if (cuda_check(h) != PLDS_OK) {
        free_all(h);
        delete h;
        set_status(PLDS_EDEVICE);
        return nullptr;
    }
    set_status(PLDS_OK);
    return h;
}

plds_t *plds_create(int32_t n, double delta, double lambda) {
    return plds_create_ex(n, delta, lambda, 0, nullptr, nullptr, 0);
}

int plds_batch_insert(plds_t *h, const int32_t *edges, int64_t B) {
    return set_status(run_op(h, edges, B, kOpInsert));
}

int plds_batch_delete(plds_t *h, const int32_t *edges, int64_t B) {
    return set_status(run_op(h, edges, B, kOpDelete));
}

static int copy_out(plds *h, void *dst, const void *src, size_t bytes) {
    if (is_device_ptr(dst)) cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->stream);
    else cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        h->poisoned = true;
        return PLDS_EDEVICE;
    }
    return PLDS_OK;
}

static int coreness_impl(plds *h, double *est, int32_t *expo) {
    if (!h) return PLDS_EINVAL;
    if (h->poisoned) return PLDS_EPOISONED;
    cudaSetDevice(h->device);
    const size_t N = (size_t)h->n;
    bool est_dev = est && is_device_ptr(est), exp_dev = expo && is_device_ptr(expo);
    DevBuf tmp_est, tmp_exp;
    double *de = est_dev ? est : nullptr;
    int32_t *dx = exp_dev ? expo : nullptr;
    if (est && !est_dev) {
        if (!dev_get(h, tmp_est, 8 * N)) return PLDS_ENOMEM;
        de = P<double>(tmp_est);
    }
    if (expo && !exp_dev) {
        if (!dev_get(h, tmp_exp, 4 * N)) {
            dev_free(h, tmp_est);
            return PLDS_ENOMEM;
        }
        dx = P<int32_t>(tmp_exp);
    }
    int blocks = std::max(1, std::min(h->num_sms * 8, (int)((h->n + 255) / 256)));
    h->launches++;
    k_coreness<<<blocks, 256, 0, h->stream>>>(P<int32_t>(h->level), P<int32_t>(h->deg), h->n, h->T.Lg,
                                              P<double>(h->powtab), de, dx);
    int rc = cuda_check(h);
    if (!rc && est && !est_dev) cudaMemcpyAsync(est, de, 8 * N, cudaMemcpyDeviceToHost, h->stream);
    if (!rc && expo && !exp_dev) cudaMemcpyAsync(expo, dx, 4 * N, cudaMemcpyDeviceToHost, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        h->poisoned = true;
        rc = PLDS_EDEVICE;
    }
    dev_free(h, tmp_est);
    dev_free(h, tmp_exp);
    return rc;
}

int plds_coreness(plds_t *h, double *out) {
    if (!out) return set_status(PLDS_EINVAL);
    return set_status(coreness_impl(h, out, nullptr));
}

int plds_coreness_exponent(plds_t *h, int32_t *out) {
    if (!out) return set_status(PLDS_EINVAL);
    return set_status(coreness_impl(h, nullptr, out));
}

// ---------------------------------------------------------------------------
// Low out-degree orientation (Section "O(alpha) Out-Degree Orientation",
// Algorithm 5): an edge goes from the endpoint on the lower level to the one on
// the higher level, on equal levels from the lower id to the higher id (the
// reading of Algorithm 5's flip conditions).  Queries on the current levels,
// and the flipped edges F and oriented updates J of the last batch call made
// with tuning.track_orientation set (levels saved at its start).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool edge_goes_from(const int32_t *lv, int32_t u, int32_t v) {
    const int32_t a = lv[u], b = lv[v];
    return a < b || (a == b && u < v);
}

__global__ void k_orient(const int32_t *level, const int32_t *slots, const int64_t *off, const int32_t *cap,
                         int32_t n, const int2 *edges, int64_t B, int32_t *tail) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < B; i += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = edges[i];
        int32_t t = -1;
        if (e.x >= 0 && e.x < n && e.y >= 0 && e.y < n && e.x != e.y && table_find(slots, off[e.x], cap[e.x], e.y))
            t = edge_goes_from(level, e.x, e.y) ? e.x : e.y;
        tail[i] = t;
    }
}

// One warp per vertex: neighbours w with v -> w.
__global__ void k_out_degrees(const int32_t *level, const int32_t *slots, const int64_t *off, const int32_t *cap,
                              int32_t n, int32_t *out) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
        const int32_t lv = level[v], c = cap[v];
        const int4 *t = reinterpret_cast<const int4 *>(slots + off[v]);
        int cnt = 0;
        for (int j = lane; j < (c >> 2); j += 32) {
            const int4 q = t[j];
            const int32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int32_t w = w4[k];
                if (w >= 0 && w < n) {
                    const int32_t lw = level[w];
                    cnt += (lv < lw || (lv == lw && (int32_t)v < w)) ? 1 : 0;
                }
            }
        }
        cnt = warp_sum(cnt);
        if (lane == 0) out[v] = cnt;
    }
}

__global__ void k_keyset_build(const unsigned long long *keys, int64_t m, unsigned long long *set, int64_t cap) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        uint64_t h = mix64(k) & (uint64_t)(cap - 1);
        for (int64_t it = 0; it < cap; ++it) {
            const unsigned long long o = atomicCAS(&set[h], kEmptyKey, k);
            if (o == kEmptyKey || o == k) break;
            h = (h + 1) & (uint64_t)(cap - 1);
        }
    }
}

__device__ __forceinline__ bool keyset_has(const unsigned long long *set, int64_t cap, unsigned long long k) {
    uint64_t h = mix64(k) & (uint64_t)(cap - 1);
    for (int64_t it = 0; it < cap; ++it) {
        const unsigned long long o = set[h];
        if (o == k) return true;
        if (o == kEmptyKey) return false;
        h = (h + 1) & (uint64_t)(cap - 1);
    }
    return false;
}

// One warp per vertex whose level changed: its edges whose orientation differs
// between the saved and the current levels (each edge once: from its lower
// endpoint among those that moved), minus the edges the batch inserted.
__global__ void k_flips(const int32_t *level, const int32_t *old_level, const int32_t *slots, const int64_t *off,
                        const int32_t *cap, int32_t n, const unsigned long long *inserted, int64_t icap, int2 *out,
                        int64_t out_cap, unsigned long long *count) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v64 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v64 < n; v64 += nw) {
        const int32_t v = (int32_t)v64;
        if (old_level[v] == level[v]) continue;
        const int32_t c = cap[v];
        const int4 *t = reinterpret_cast<const int4 *>(slots + off[v]);
        for (int j = lane; j < (c >> 2); j += 32) {
            const int4 q = t[j];
            const int32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int32_t w = w4[k];
                if (w < 0 || w >= n) continue;
                if (w < v && old_level[w] != level[w]) continue;
                const bool b = edge_goes_from(old_level, v, w), a = edge_goes_from(level, v, w);
                if (a == b) continue;
                if (icap > 0) {
                    const unsigned long long key =
                        ((unsigned long long)(uint32_t)min(v, w) << 32) | (uint32_t)max(v, w);
                    if (keyset_has(inserted, icap, key)) continue;
                }
                const unsigned long long pos = atomicAdd(count, 1ull);
                if ((int64_t)pos < out_cap) out[pos] = b ? make_int2(v, w) : make_int2(w, v);
            }
        }
    }
}

__global__ void k_oriented_updates(const unsigned long long *keys, int64_t m, const int32_t *lv, int2 *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = (int32_t)(keys[i] >> 32), v = (int32_t)(keys[i] & 0xffffffffull);
        out[i] = edge_goes_from(lv, u, v) ? make_int2(u, v) : make_int2(v, u);
    }
}

static int orient_grid(const plds *h) { return h->num_sms * 8; }

int plds_orient(plds_t *h, const int32_t *edges, int64_t B, int32_t *tail) {
    if (!h || B < 0 || (B > 0 && (!edges || !tail))) return set_status(PLDS_EINVAL);
    if (h->poisoned) return set_status(PLDS_EPOISONED);
    if (B == 0) return set_status(PLDS_OK);
    cudaSetDevice(h->device);
    const bool din = is_device_ptr(edges), dout = is_device_ptr(tail);
    const size_t ebytes = sizeof(int2) * (size_t)B, tbytes = sizeof(int32_t) * (size_t)B;
    if (!dev_get(h, h->oscratch, (din ? 0 : ebytes) + (dout ? 0 : tbytes) + 16)) return set_status(PLDS_ENOMEM);
    unsigned char *scr = P<unsigned char>(h->oscratch);
    const int2 *de = din ? reinterpret_cast<const int2 *>(edges) : reinterpret_cast<const int2 *>(scr);
    int32_t *dt = dout ? tail : reinterpret_cast<int32_t *>(scr + (din ? 0 : ebytes));
    if (!din) cudaMemcpyAsync(scr, edges, ebytes, cudaMemcpyHostToDevice, h->stream);
    k_orient<<<orient_grid(h), 256, 0, h->stream>>>(P<int32_t>(h->level), P<int32_t>(h->pool), P<int64_t>(h->off),
                                                    P<int32_t>(h->cap), h->n, de, B, dt);
    h->launches++;
    if (!dout) cudaMemcpyAsync(tail, dt, tbytes, cudaMemcpyDeviceToHost, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        h->poisoned = true;
        return set_status(PLDS_EDEVICE);
    }
    return set_status(PLDS_OK);
}

int plds_out_degrees(plds_t *h, int32_t *out) {
    if (!h || !out) return set_status(PLDS_EINVAL);
    if (h->poisoned) return set_status(PLDS_EPOISONED);
    cudaSetDevice(h->device);
    const bool dout = is_device_ptr(out);
    if (!dout && !dev_get(h, h->oscratch, 4 * (size_t)h->n)) return set_status(PLDS_ENOMEM);
    int32_t *d = dout ? out : P<int32_t>(h->oscratch);
    k_out_degrees<<<orient_grid(h), 256, 0, h->stream>>>(P<int32_t>(h->level), P<int32_t>(h->pool), P<int64_t>(h->off),
                                                         P<int32_t>(h->cap), h->n, d);
    h->launches++;
    if (!dout) cudaMemcpyAsync(out, d, 4 * (size_t)h->n, cudaMemcpyDeviceToHost, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        h->poisoned = true;
        return set_status(PLDS_EDEVICE);
    }
    return set_status(PLDS_OK);
}

// Copies up to cap pairs of a device list of `total` pairs to out (host or device).
static int pairs_out(plds *h, int32_t *out, int64_t cap, const void *src, int64_t total) {
    const int64_t k = std::min(cap, total);
    if (k > 0 && out) {
        const size_t bytes = sizeof(int2) * (size_t)k;
        cudaMemcpyAsync(out, src, bytes, is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        h->stream);
    }
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        h->poisoned = true;
        return PLDS_EDEVICE;
    }
    return PLDS_OK;
}

int plds_flips(plds_t *h, int32_t *out, int64_t cap, int64_t *count) {
    if (!h || !count || cap < 0 || (cap > 0 && !out)) return set_status(PLDS_EINVAL);
    if (h->poisoned) return set_status(PLDS_EPOISONED);
    if (!h->orient_ok) return set_status(PLDS_EINVAL);  // tracking off, or another call since the batch
    cudaSetDevice(h->device);
    const int64_t m = (int64_t)h->host_ctl.vcount;
    int64_t icap = 0;
    if (h->orient_op == kOpInsert && m > 0) {  // the batch's inserted edges are not flips
        icap = pow2_at_least(2 * m);
        if (!dev_get(h, h->okeys, 8 * (size_t)icap)) return set_status(PLDS_ENOMEM);
        cudaMemsetAsync(h->okeys.p, 0xff, 8 * (size_t)icap, h->stream);
        k_keyset_build<<<orient_grid(h), 256, 0, h->stream>>>(P<unsigned long long>(h->vkeys), m,
                                                               P<unsigned long long>(h->okeys), icap);
        h->launches++;
    }
    // count first, then collect into scratch sized by the count
    int64_t total = 0;
    for (int pass = 0; pass < 2; ++pass) {
        const int64_t want = pass == 0 ? 0 : total;
        if (!dev_get(h, h->oscratch, 8 + sizeof(int2) * (size_t)want + 16)) return set_status(PLDS_ENOMEM);
        unsigned long long *cnt = P<unsigned long long>(h->oscratch);
        int2 *lst = reinterpret_cast<int2 *>(P<unsigned char>(h->oscratch) + 16);
        cudaMemsetAsync(cnt, 0, 8, h->stream);
        k_flips<<<orient_grid(h), 256, 0, h->stream>>>(P<int32_t>(h->level), P<int32_t>(h->old_level),
                                                       P<int32_t>(h->pool), P<int64_t>(h->off), P<int32_t>(h->cap),
                                                       h->n, P<unsigned long long>(h->okeys), icap, lst, want, cnt);
        h->launches++;
        unsigned long long c = 0;
        cudaMemcpyAsync(&c, cnt, 8, cudaMemcpyDeviceToHost, h->stream);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
            cudaGetLastError();
            h->poisoned = true;
            return set_status(PLDS_EDEVICE);
        }
        total = (int64_t)c;
        if (pass == 1 || total == 0 || cap == 0) break;
    }
    *count = total;
    if (total > 0 && cap > 0) {
        const int rc = pairs_out(h, out, cap, P<unsigned char>(h->oscratch) + 16, total);
        if (rc) return set_status(rc);
    }
    return set_status(PLDS_OK);
}

int plds_oriented_updates(plds_t *h, int32_t *out, int64_t cap, int64_t *count) {
    if (!h || !count || cap < 0 || (cap > 0 && !out)) return set_status(PLDS_EINVAL);
    if (h->poisoned) return set_status(PLDS_EPOISONED);
    if (!h->orient_ok) return set_status(PLDS_EINVAL);
    cudaSetDevice(h->device);
    const int64_t m = (int64_t)h->host_ctl.vcount;
    *count = m;
    if (m == 0 || cap == 0) return set_status(PLDS_OK);
    if (!dev_get(h, h->oscratch, sizeof(int2) * (size_t)m + 16)) return set_status(PLDS_ENOMEM);
    int2 *lst = reinterpret_cast<int2 *>(P<unsigned char>(h->oscratch));
    const int32_t *lv = h->orient_op == kOpInsert ? P<int32_t>(h->level) : P<int32_t>(h->old_level);
    k_oriented_updates<<<orient_grid(h), 256, 0, h->stream>>>(P<unsigned long long>(h->vkeys), m, lv, lst);
    h->launches++;
    return set_status(pairs_out(h, out, cap, lst, m));
}

// ---------------------------------------------------------------------------
// Static (2+eps')-approximate k-core (Section "Static (2+eps)-Approximate k-Core",
// Algorithm 6) on the handle's current graph, without touching its levels: one
// cooperative kernel, three grid-barrier phases per peeling iteration -- select
// (peel the lowest bucket, compact the survivors), count (each peeled vertex's
// surviving neighbours: r_v by atomics), update (over all survivors: those with
// r_v > 0 get C = max(C - r, ceil((1+eps)^(t-1))) and bucket = max(bucket(C), t);
// every survivor's bucket enters the minimum that picks the next bucket).  Buckets are decided by comparing integers with the
// host-built table thr[b] = (1+eps)^b, so the estimates thr[bucket when peeled]
// are exact copies of the table's doubles.
// ---------------------------------------------------------------------------
namespace {
struct StaticCtl {
    unsigned long long bar_arrivals;  // grid barrier (same layout as Ctl's first word)
    int32_t err;
    int32_t acnt[2];    // alive lists
    int32_t icnt;       // peeled in this iteration
    int32_t minb[3];    // lowest bucket among survivors (per iteration mod 3)
    unsigned long long outer, inner, visits;
};
struct StaticArgs {
    int32_t n, nb, J;
    const int32_t *deg, *cap;
    const int64_t *off;
    const int32_t *slots;
    const double *thr, *lim;
    const int32_t *floor_c;
    int32_t *C, *bk, *r, *A0, *A1, *I;
    double *est;
    StaticCtl *sc;
    int64_t wait_limit_ns;
};
}  // namespace

__device__ __forceinline__ int32_t sk_bucket(const double *thr, int32_t nb, int32_t c) {
    int32_t lo = 0, hi = nb - 1;  // the smallest b with thr[b] >= c (thr is increasing)
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (thr[mid] >= (double)c) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__global__ void __launch_bounds__(512) k_static_core(const StaticArgs a) {
    GridTeam T{reinterpret_cast<Ctl *>(a.sc), a.wait_limit_ns, 32};
    StaticCtl *sc = a.sc;
    const int lane = threadIdx.x & 31;
    unsigned long long visits = 0;
    // init: C = deg, bucket of C, alive list; isolated vertices get 0
    for (int64_t v = T.tid(); v < a.n; v += T.nthreads()) {
        const int32_t d = a.deg[v];
        a.C[v] = d;
        a.r[v] = 0;
        a.est[v] = 0.0;
        int32_t b = -1;
        if (d > 0) {
            b = sk_bucket(a.thr, a.nb, d);
            a.A0[atomicAdd(&sc->acnt[0], 1)] = (int32_t)v;
            atomicMin(&sc->minb[0], b);
        }
        a.bk[v] = b;
    }
    if (!T.sync()) return;
    int32_t t = ld_volatile(&sc->minb[0]), bkt = t, j = 0;
    for (int it = 1;; ++it) {
        if (ld_volatile(&sc->acnt[(it - 1) & 1]) == 0) break;
        const int cur = (it - 1) & 1, nxt = it & 1, w = it % 3;
        const int32_t ac = ld_volatile(&sc->acnt[cur]);
        const int32_t *A = cur ? a.A1 : a.A0;
        int32_t *An = nxt ? a.A1 : a.A0;
        if (T.leader()) {
            sc->minb[(it + 1) % 3] = 0x7fffffff;  // written in iteration it + 1, last read two barriers ago
            sc->inner += 1;
            if (j == 0) sc->outer += 1;
        }
        // select: peel bucket bkt, keep the rest
        for (int64_t i0 = (int64_t)T.wid() * 32; i0 < ac; i0 += (int64_t)T.nwarps() * 32) {
            const int64_t i = i0 + lane;
            int32_t v = 0, b = -1;
            if (i < ac) {
                v = A[i];
                b = a.bk[v];
            }
            const bool peel = i < ac && b == bkt, keep = i < ac && b != bkt;
            if (peel) {
                a.bk[v] = -1;
                a.est[v] = a.thr[bkt];
            }
            const int pi = warp_append(&sc->icnt, peel);
            if (peel) a.I[pi] = v;
            const int pk = warp_append(&sc->acnt[nxt], keep);
            if (keep) An[pk] = v;
        }
        if (!T.sync()) return;
        // count: surviving neighbours of the peeled vertices
        const int32_t ic = ld_volatile(&sc->icnt);
        if (T.leader()) sc->acnt[cur] = 0;  // read by every thread before the barrier
        for (int64_t i = T.wid(); i < ic; i += T.nwarps()) {
            const int32_t u = a.I[i];
            const int4 *tb = reinterpret_cast<const int4 *>(a.slots + a.off[u]);
            const int32_t ng = a.cap[u] >> 2;
            for (int32_t g0 = 0; g0 < ng; g0 += 32) {
                const int32_t gi = g0 + lane;
                const int4 q = gi < ng ? tb[gi] : make_int4(-1, -1, -1, -1);
                const int32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int32_t x = w4[k];
                    if (x >= 0 && x < a.n) {
                        ++visits;
                        if (a.bk[x] >= 0) atomicAdd(&a.r[x], 1);
                    }
                }
            }
        }
        if (!T.sync()) return;
        // update: the survivors that lost neighbours; the lowest bucket of all survivors
        const int32_t sn = ld_volatile(&sc->acnt[nxt]);
        if (T.leader()) sc->icnt = 0;
        int32_t mu = 0x7fffffff;
        for (int64_t i = T.tid(); i < sn; i += T.nthreads()) {
            const int32_t x = An[i];
            const int32_t rx = a.r[x];
            int32_t b = a.bk[x];
            if (rx > 0) {
                const int32_t c = max(a.C[x] - rx, a.floor_c[t]);
                a.C[x] = c;
                a.r[x] = 0;
                b = max(sk_bucket(a.thr, a.nb, c), t);
                a.bk[x] = b;
            }
            mu = min(mu, b);
        }
        mu = (int32_t)__reduce_min_sync(kFull, (unsigned)mu);
        if (lane == 0 && mu != 0x7fffffff) atomicMin(&sc->minb[w], mu);
        if (!T.sync()) return;
        // next: another bucket at the same threshold t while it is within (2+eps) thr[t]
        if (ld_volatile(&sc->acnt[nxt]) == 0) break;
        const int32_t next = ld_volatile(&sc->minb[w]);
        if (next < 0 || next >= a.nb) {
            if (T.leader()) {
                atomicOr(&sc->err, kErrInternal);
            }
            return;
        }
        if (j + 1 < a.J && a.thr[next] <= a.lim[t]) {
            bkt = next;
            ++j;
        } else {
            t = next;
            bkt = next;
            j = 0;
        }
    }
    visits = warp_sum64(visits);
    if (lane == 0 && visits) atomicAdd(&sc->visits, visits);
}

int plds_static_coreness(plds_t *h, double eps_prime, double *out, int64_t *stats) {
    if (!h || !out) return set_status(PLDS_EINVAL);
    if (h->poisoned) return set_status(PLDS_EPOISONED);
    StaticTables tb;
    if (build_static_tables(h->n, eps_prime, &tb) != 0) return set_status(PLDS_EINVAL);
    cudaSetDevice(h->device);
    const size_t N = (size_t)h->n, nb = tb.thr.size();
    const bool dout = is_device_ptr(out);
    if (!dev_get(h, h->sk_scratch, 4 * N * 6 + (dout ? 0 : 8 * N) + 64) ||
        !dev_get(h, h->sk_tables, 16 * nb + 4 * nb + 64) || !dev_get(h, h->sk_ctl, sizeof(StaticCtl)))
        return set_status(PLDS_ENOMEM);
    std::vector<unsigned char> host(16 * nb + 4 * nb);
    std::memcpy(host.data(), tb.thr.data(), 8 * nb);
    std::memcpy(host.data() + 8 * nb, tb.lim.data(), 8 * nb);
    std::memcpy(host.data() + 16 * nb, tb.floor_c.data(), 4 * nb);
    cudaMemcpyAsync(h->sk_tables.p, host.data(), host.size(), cudaMemcpyHostToDevice, h->stream);
    StaticCtl c0{};
    c0.minb[0] = c0.minb[1] = c0.minb[2] = 0x7fffffff;
    cudaMemcpyAsync(h->sk_ctl.p, &c0, sizeof(c0), cudaMemcpyHostToDevice, h->stream);
    int32_t *w = P<int32_t>(h->sk_scratch);
    StaticArgs a{};
    a.n = h->n;
    a.nb = (int32_t)nb;
    a.J = tb.J;
    a.deg = P<int32_t>(h->deg);
    a.cap = P<int32_t>(h->cap);
    a.off = P<int64_t>(h->off);
    a.slots = P<int32_t>(h->pool);
    a.thr = P<double>(h->sk_tables);
    a.lim = a.thr + nb;
    a.floor_c = reinterpret_cast<const int32_t *>(a.thr + 2 * nb);
    a.C = w;
    a.bk = w + N;
    a.r = w + 2 * N;
    a.A0 = w + 3 * N;
    a.A1 = w + 4 * N;
    a.I = w + 5 * N;
    a.est = dout ? out : reinterpret_cast<double *>(P<unsigned char>(h->sk_scratch) + ((4 * N * 6 + 15) & ~(size_t)15));
    a.sc = P<StaticCtl>(h->sk_ctl);
    a.wait_limit_ns = h->wait_limit_ns;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_static_core, 512, 0);
    if (occ < 1) return set_status(PLDS_EDEVICE);
    void *args[] = {(void *)&a};
    if (cudaLaunchCooperativeKernel((const void *)k_static_core, dim3(h->num_sms), dim3(512), args, 0, h->stream) !=
        cudaSuccess) {
        cudaGetLastError();
        return set_status(PLDS_EDEVICE);
    }
    h->launches++;
    StaticCtl c{};
    cudaMemcpyAsync(&c, h->sk_ctl.p, sizeof(c), cudaMemcpyDeviceToHost, h->stream);
    if (!dout) cudaMemcpyAsync(out, a.est, 8 * N, cudaMemcpyDeviceToHost, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        h->poisoned = true;
        return set_status(PLDS_EDEVICE);
    }
    if (c.err & kErrTimeout) {
        h->poisoned = true;
        return set_status(PLDS_ETIMEOUT);
    }
    if (c.err) return set_status(PLDS_EINTERNAL);
    if (stats) {
        stats[0] = (int64_t)c.outer;
        stats[1] = (int64_t)c.inner;
        stats[2] = (int64_t)c.visits;
    }
    return set_status(PLDS_OK);
}

int plds_levels(plds_t *h, int32_t *out) {
    if (!h || !out) return set_status(PLDS_EINVAL);
    if (h->poisoned) return set_status(PLDS_EPOISONED);
    return set_status(copy_out(h, out, h->level.p, 4 * (size_t)h->n));
}

int plds_counters(plds_t *h, int32_t *deg, int32_t *up, int32_t *upstar) {
    if (!h) return set_status(PLDS_EINVAL);
    if (h->poisoned) return set_status(PLDS_EPOISONED);
    const size_t bytes = 4 * (size_t)h->n;
    int rc = PLDS_OK;
    if (deg && !rc) rc = copy_out(h, deg, h->deg.p, bytes);
    if (up && !rc) rc = copy_out(h, up, h->up.p, bytes);
    if (upstar && !rc) rc = copy_out(h, upstar, h->upstar.p, bytes);
    return set_status(rc);
}

int plds_stats(plds_t *h, plds_stats_t *out) {
    if (!h || !out) return set_status(PLDS_EINVAL);
    unsigned long long top = 0;
    cudaMemcpyAsync(&top, h->pool_top.p, 8, cudaMemcpyDeviceToHost, h->stream);
    cudaStreamSynchronize(h->stream);
    *out = h->last;
    out->pool_slots_used = (int64_t)top;
    out->pool_slots_cap = h->pool_cap;
    out->device_bytes = h->device_bytes;
    out->pool_grows = h->pool_grows;
    out->launches = h->launches;
    return set_status(PLDS_OK);
}

int plds_params(plds_t *h, int32_t *out) {
    if (!h || !out) return set_status(PLDS_EINVAL);
    out[0] = h->T.t;
    out[1] = h->T.Lg;
    out[2] = h->T.G;
    out[3] = h->T.K;
    return set_status(PLDS_OK);
}

int plds_tables(plds_t *h, int32_t *upmax, int32_t *dnmin) {
    if (!h) return set_status(PLDS_EINVAL);
    if (upmax) std::memcpy(upmax, h->T.upmax.data(), 4 * (size_t)h->T.G);
    if (dnmin) std::memcpy(dnmin, h->T.dnmin.data(), 4 * (size_t)h->T.G);
    return set_status(PLDS_OK);
}

int plds_set_stream(plds_t *h, void *stream) {
    if (!h) return set_status(PLDS_EINVAL);
    cudaStreamSynchronize(h->stream);
    h->stream = (cudaStream_t)stream;
    return set_status(PLDS_OK);
}

int plds_set_tuning(plds_t *h, const plds_tuning *t) {
    if (!h || !t) return set_status(PLDS_EINVAL);
    if (t->block_threads && (t->block_threads % 32 || t->block_threads < 128 || t->block_threads > 512))
        return set_status(PLDS_EINVAL);
    if (t->thread_max_cap < 0 || t->load_num < 0 || t->load_den < 0 || t->blocks_per_sm < 0 ||
        t->test_delay_us < 0 || t->test_delay_us > 10 * 1000 * 1000 || t->barrier_sleep_ns < -1 ||
        t->barrier_sleep_ns > 100000 || t->block_cap < 0 || (t->block_cap > 0 && t->block_cap < 4) ||
        t->list_cap < 0)
        return set_status(PLDS_EINVAL);
    if ((t->load_num > 0) != (t->load_den > 0) || (t->load_num > 0 && (t->load_num * 8 > t->load_den * 7)))
        return set_status(PLDS_EINVAL);  // a table must keep an empty slot
    if (t->trace_rounds && !dev_get(h, h->trace, 48 * ((size_t)h->T.K + 16))) return set_status(PLDS_ENOMEM);
    h->tune = *t;
    return set_status(PLDS_OK);
}

int plds_set_wait_limit(plds_t *h, int64_t ns) {
    if (!h || ns < 0) return set_status(PLDS_EINVAL);
    h->wait_limit_ns = ns > 0 ? ns : 20ll * 1000 * 1000 * 1000;
    return set_status(PLDS_OK);
}

int plds_trace(plds_t *h, int32_t *out, int32_t cap) {
    if (!h || !out || cap < 0) return set_status(PLDS_EINVAL);
    if (!h->tune.trace_rounds || !h->trace.p) return set_status(0);
    int32_t k = std::min<int32_t>(h->host_ctl.trace_n, std::min<int32_t>(cap, (int32_t)(h->trace.bytes / 48)));
    if (k > 0) cudaMemcpy(out, h->trace.p, 48 * (size_t)k, cudaMemcpyDeviceToHost);
    set_status(PLDS_OK);
    return k;
}

int plds_last_status(void) { return g_last_status; }

void plds_destroy(plds_t *h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    free_all(h);
    cudaStreamSynchronize(h->stream);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->evm) cudaEventDestroy(h->evm);
    cudaGetLastError();
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batch entry point.
//
// Some callers must not allocate device memory while they apply updates: a
// latency-critical update loop cannot afford cudaMalloc (it may synchronise the
// whole device and stall every stream), and a process that runs under a fixed
// device-memory budget, or whose allocator belongs to a host framework that
// cannot be re-entered from this call, has no allocator to lend.  For them,
// plds_batch_static applies a batch using only memory that already exists: the
// handle's own arrays (allocated by plds_create*) and one file-scope device
// array that holds the per-batch scratch (edge staging, key set, key lists,
// touched and candidate lists, shrink scratch) for batches of at most
// kStaticMaxB edges.  The array costs every GPU that loads this library 4 MiB
// until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t kStaticMaxB = 1 << 16;         // edges per call
constexpr int64_t kStaticHcap = 1 << 17;         // key-set entries (power of two >= 2 * kStaticMaxB)
constexpr int64_t kStaticTcap = 2 * kStaticMaxB;  // touched vertices / sorted candidates
constexpr int64_t kStaticArena = 1 << 17;        // ints of table-shrink scratch
constexpr size_t kStOffEdges = 0;
constexpr size_t kStOffHset = kStOffEdges + 8 * (size_t)kStaticMaxB;
constexpr size_t kStOffUkeys = kStOffHset + 8 * (size_t)kStaticHcap;
constexpr size_t kStOffVkeys = kStOffUkeys + 8 * (size_t)kStaticMaxB;
constexpr size_t kStOffTouched = kStOffVkeys + 8 * (size_t)kStaticMaxB;
constexpr size_t kStOffS = kStOffTouched + 4 * (size_t)kStaticTcap;
constexpr size_t kStOffArena = kStOffS + 4 * (size_t)kStaticTcap;
constexpr size_t kStaticBytes = kStOffArena + 4 * (size_t)kStaticArena;  // 4 MiB
constexpr int kMaxDevices = 128;
}  // namespace

// Shared by every call on a device; it keeps the previous call's contents.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

static std::mutex g_static_mu;
static unsigned char *g_static_addr[kMaxDevices];

// Device address of g_static_scratch on the current device (looked up once per
// device; in host code the symbol itself is only a host-side stand-in).  The
// address belongs to the device's context: after cudaDeviceReset it is stale, as
// is every handle created before the reset.
static unsigned char *static_scratch(int device) {
    if (device < 0 || device >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[device]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_static_addr[device] = static_cast<unsigned char *>(p);
    }
    return g_static_addr[device];
}

extern "C" int plds_batch_static(plds_t *h, const int32_t *edges, int64_t B, int32_t is_delete) {
    if (!h || B < 0 || (B > 0 && !edges) || (is_delete != 0 && is_delete != 1)) return set_status(PLDS_EINVAL);
    if (B > kStaticMaxB) return set_status(PLDS_EINVAL);  // larger batches need plds_batch_insert/delete
    if (h->poisoned) return set_status(PLDS_EPOISONED);
    std::memset(&h->last, 0, sizeof(h->last));
    h->last.submitted = B;
    h->orient_ok = false;
    if (B == 0) return set_status(PLDS_OK);
    if (cudaSetDevice(h->device) != cudaSuccess) {
        cudaGetLastError();
        return set_status(PLDS_EDEVICE);
    }
    unsigned char *base = static_scratch(h->device);
    if (!base) return set_status(PLDS_EDEVICE);
    const int32_t op = is_delete ? kOpDelete : kOpInsert;
    const int32_t *dedges = edges;
    if (!is_device_ptr(edges)) {
        cudaMemcpyAsync(base + kStOffEdges, edges, sizeof(int32_t) * 2 * (size_t)B, cudaMemcpyHostToDevice,
                        h->stream);
        dedges = reinterpret_cast<const int32_t *>(base + kStOffEdges);
    }
    if ((int64_t)h->stamp_base + 2 * (int64_t)h->T.K + 8 >= 0x7fffffff) {
        cudaMemsetAsync(h->stamp.p, 0, sizeof(int32_t) * (size_t)h->n, h->stream);
        h->stamp_base = 1;
    }
    // what must start empty: control words, the key set (as large as the batch
    // needs: a power of two >= 2B, so small batches clear little), the level histogram
    const int64_t hc = std::min<int64_t>(kStaticHcap, pow2_at_least(2 * std::max<int64_t>(B, 1024)));
    cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), h->stream);
    cudaMemsetAsync(base + kStOffHset, 0xff, 8 * (size_t)hc, h->stream);
    if (op == kOpInsert) cudaMemsetAsync(h->bins.p, 0, sizeof(int32_t) * ((size_t)h->T.K + 1), h->stream);
    GraphCtx g = make_ctx(h, op, dedges, B);
    g.hset = reinterpret_cast<unsigned long long *>(base + kStOffHset);
    g.hcap = hc;
    g.ukeys = reinterpret_cast<unsigned long long *>(base + kStOffUkeys);
    g.vkeys = reinterpret_cast<unsigned long long *>(base + kStOffVkeys);
    g.touched = reinterpret_cast<int32_t *>(base + kStOffTouched);
    g.S = reinterpret_cast<int32_t *>(base + kStOffS);
    g.arena = reinterpret_cast<int32_t *>(base + kStOffArena);
    g.arena_cap = kStaticArena;
    h->stamp_base += h->T.K + 2;
    launch_pre(h, g);
    int rc = launch_batch(h, g);
    if (rc) return set_status(rc);
    cudaMemcpyAsync(&h->host_ctl, h->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream);
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        h->poisoned = true;
        return set_status(PLDS_EDEVICE);
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess) h->last.kernel_ns = (int64_t)(ms * 1e6);
    if (cudaEventElapsedTime(&ms, h->ev0, h->evm) == cudaSuccess) h->last.pre_ns = (int64_t)(ms * 1e6);
    cudaGetLastError();
    const Ctl &c = h->host_ctl;
    h->last.err_bits = c.err;
    h->last.err_site = c.err_site;
    h->last.err_info[0] = c.err_info[0];
    h->last.err_info[1] = c.err_info[1];
    h->last.err_info[2] = c.err_info[2];
    if (c.err & kErrTimeout) {
        h->poisoned = true;
        return set_status(PLDS_ETIMEOUT);
    }
    if (c.err & kErrInvalidId) {
        undo_incoming(h, c, g);
        return set_status(PLDS_EINVAL);
    }
    // the adjacency pool is full: growing it would allocate, so report and leave
    // the graph unchanged (a regular plds_batch_insert call can grow it)
    if (c.err == kErrNeedPool) return set_status(PLDS_ENOMEM);
    if (c.err) {
        h->poisoned = true;
        return set_status(PLDS_EINTERNAL);
    }
    h->last.self_loops = (int64_t)c.st[kStSelfLoops];
    h->last.duplicates = B - h->last.self_loops - (int64_t)c.ucount;
    h->last.filtered = (int64_t)c.st[kStFiltered];
    h->last.valid = (int64_t)c.vcount;
    h->last.rounds = (int64_t)c.st[kStRounds];
    h->last.moves = (int64_t)c.st[kStMoves];
    h->last.visits = (int64_t)c.st[kStVisits];
    h->last.dl_evals = (int64_t)c.st[kStDlEvals];
    h->last.dl_visits = (int64_t)c.st[kStDlVisits];
    h->last.slots_scanned = (int64_t)c.st[kStSlotsScanned];
    h->last.up_visits = (int64_t)c.st[kStUpVisits];
    h->last.affected = (int64_t)c.st[kStAffected];
    h->last.skipped_rounds = (int64_t)c.st[kStSkipRounds];
    h->last.skipped_moves = (int64_t)c.st[kStSkipMoves];
    h->last.skipped_visits = (int64_t)c.st[kStSkipVisits];
    h->last.skipped_up_visits = (int64_t)c.st[kStSkipUpVisits];
    return set_status(PLDS_OK);
}

// ---------------------------------------------------------------------------
// Batched form: many independent graphs, one launch per round of batches.
//
// A set owns `count` ordinary handles.  One round applies one mixed batch to
// every graph (its insertion half, then its deletion half, as Algorithm 1
// orders them).  The kernel is persistent: each block takes the next graph from
// a work counter (graphs ordered by decreasing size) and runs that graph's whole
// round with the same device routines as the single-graph kernel, the block
// being the team (block barriers only, graphs progress independently).  The
// per-round launch sequence (descriptor upload, counter reset, kernel, control
// word read-back) is captured once in a CUDA graph and replayed.
// ---------------------------------------------------------------------------
namespace {
struct SetItem {
    GraphCtx half[2];  // 0: insertion half, 1: deletion half
};
constexpr int kSetThreads = 256;
constexpr int kSetStageShift = 3;
}  // namespace

__global__ void __launch_bounds__(kSetThreads, 2)
    k_batch_set(const SetItem *__restrict__ items, int32_t count, int32_t *next) {
    extern __shared__ int32_t sh[];
    __shared__ GraphCtx gsh;
    __shared__ int32_t idx;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) idx = atomicAdd(next, 1);
        __syncthreads();
        const int i = idx;
        if (i >= count) return;
        for (int h = 0; h < 2; ++h) {
            __syncthreads();
            const int32_t *src = reinterpret_cast<const int32_t *>(&items[i].half[h]);
            int32_t *dst = reinterpret_cast<int32_t *>(&gsh);
            for (int k = threadIdx.x; k < (int)(sizeof(GraphCtx) / 4); k += blockDim.x) dst[k] = src[k];
            __syncthreads();
            // the host reads both halves' control blocks: clear them even for an empty half
            int32_t *cw = reinterpret_cast<int32_t *>(gsh.ctl);
            for (int k = threadIdx.x; k < (int)(sizeof(Ctl) / 4); k += blockDim.x) cw[k] = 0;
            if (gsh.B == 0) continue;  // an empty half changes nothing
            for (int64_t k = threadIdx.x; k < gsh.hcap; k += blockDim.x) gsh.hset[k] = kEmptyKey;
            if (gsh.op == kOpInsert)
                for (int k = threadIdx.x; k <= gsh.K; k += blockDim.x) gsh.bins[k] = 0;
            __syncthreads();
            BlockTeam T{gsh.ctl};
            run_batch(T, gsh, BatchIn{gsh.edges, gsh.B, gsh.op, gsh.stamp_base}, sh, kSetStageShift);
            __syncthreads();
            if (ld_volatile(&gsh.ctl->err) != 0) break;  // the host resolves it and reruns this graph
        }
    }
}

struct plds_set {
    int32_t count = 0;
    std::vector<plds *> g;       // graph handles
    std::vector<int32_t> order;  // graphs by decreasing n
    cudaStream_t stream = nullptr;   // the caller's stream (allocations, copies)
    cudaStream_t run = nullptr;      // private stream the captured round is replayed on
    bool graph_ok = true;
    plds *owner = nullptr;       // allocator and device of the set's own buffers
    DevBuf items, ctls, next, edges;
    int64_t edges_cap = 0;
    SetItem *h_items = nullptr;  // pinned
    Ctl *h_ctls = nullptr;       // pinned
    int grid = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t captured_count = -1;
    // what plds_set_create was given (the autotuner builds scratch sets alike)
    std::vector<int32_t> ns;
    double delta = 0, lambda = 0;
    plds_allocator alloc{};
    bool has_alloc = false;
};

// Runs one round for n_items graphs on the private stream (the caller's stream
// has been synchronised, so everything it enqueued before is visible).
static int set_launch(plds_set *s, int32_t n_items, bool use_graph) {
    const size_t smem = smem_bytes(kSetThreads, kSetStageShift);
    cudaStream_t st = s->run;
    use_graph = use_graph && s->graph_ok;
    if (use_graph && s->exec && s->captured_count == n_items) return cudaGraphLaunch(s->exec, st) == cudaSuccess ? 0 : -1;
    auto enqueue = [&]() {
        cudaMemcpyAsync(s->items.p, s->h_items, sizeof(SetItem) * (size_t)n_items, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(s->next.p, 0, sizeof(int32_t), st);
        k_batch_set<<<s->grid, kSetThreads, smem, st>>>(P<SetItem>(s->items), n_items, P<int32_t>(s->next));
        cudaMemcpyAsync(s->h_ctls, s->ctls.p, sizeof(Ctl) * 2 * (size_t)n_items, cudaMemcpyDeviceToHost, st);
    };
    if (!use_graph) {
        enqueue();
        return cudaGetLastError() == cudaSuccess ? 0 : -1;
    }
    if (s->exec) {
        cudaGraphExecDestroy(s->exec);
        s->exec = nullptr;
    }
    if (s->graph) {
        cudaGraphDestroy(s->graph);
        s->graph = nullptr;
    }
    bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        enqueue();
        ok = cudaStreamEndCapture(st, &s->graph) == cudaSuccess &&
             cudaGraphInstantiate(&s->exec, s->graph, 0) == cudaSuccess;
    }
    if (!ok) {  // capture unavailable: launch directly from now on
        cudaGetLastError();
        s->graph_ok = false;
        enqueue();
        return cudaGetLastError() == cudaSuccess ? 0 : -1;
    }
    s->captured_count = n_items;
    return cudaGraphLaunch(s->exec, st) == cudaSuccess ? 0 : -1;
}

extern "C" plds_set_t *plds_set_create(int32_t count, const int32_t *n, double delta, double lambda,
                                       const plds_allocator *allocator, void *stream) {
    if (count <= 0 || !n) {
        set_status(PLDS_EINVAL);
        return nullptr;
    }
    plds_set *s = new (std::nothrow) plds_set();
    if (!s) {
        set_status(PLDS_ENOMEM);
        return nullptr;
    }
    s->count = count;
    s->stream = (cudaStream_t)stream;
    s->ns.assign(n, n + count);
    s->delta = delta;
    s->lambda = lambda;
    if (allocator) {
        s->alloc = *allocator;
        s->has_alloc = true;
    }
    for (int32_t i = 0; i < count; ++i) {
        plds_t *h = plds_create_ex(n[i], delta, lambda, 0, allocator, stream, 0);
        if (!h) {
            int rc = plds_last_status();
            plds_set_destroy(s);
            set_status(rc);
            return nullptr;
        }
        // one block per graph: tables up to 64 slots are scanned better by one thread,
        // and a whole block pays off only for tables above 4096 slots
        h->tune.thread_max_cap = 64;
        h->tune.block_cap = 4096;
        s->g.push_back(h);
    }
    s->owner = s->g[0];
    if (cudaStreamCreateWithFlags(&s->run, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        plds_set_destroy(s);
        set_status(PLDS_EDEVICE);
        return nullptr;
    }
    s->order.resize(count);
    for (int32_t i = 0; i < count; ++i) s->order[i] = i;
    std::stable_sort(s->order.begin(), s->order.end(), [&](int a, int b) { return s->g[a]->n > s->g[b]->n; });
    if (!dev_get(s->owner, s->items, sizeof(SetItem) * (size_t)count) ||
        !dev_get(s->owner, s->ctls, sizeof(Ctl) * 2 * (size_t)count) || !dev_get(s->owner, s->next, 16) ||
        cudaMallocHost(&s->h_items, sizeof(SetItem) * (size_t)count) != cudaSuccess ||
        cudaMallocHost(&s->h_ctls, sizeof(Ctl) * 2 * (size_t)count) != cudaSuccess) {
        cudaGetLastError();
        plds_set_destroy(s);
        set_status(PLDS_ENOMEM);
        return nullptr;
    }
    const size_t smem = smem_bytes(kSetThreads, kSetStageShift);
    cudaFuncSetAttribute(k_batch_set, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_set, kSetThreads, smem);
    s->grid = std::max(1, occ) * s->owner->num_sms;
    set_status(PLDS_OK);
    return s;
}

extern "C" plds_t *plds_set_graph(plds_set_t *s, int32_t i) {
    if (!s || i < 0 || i >= s->count) {
        set_status(PLDS_EINVAL);
        return nullptr;
    }
    set_status(PLDS_OK);
    return s->g[i];
}

extern "C" int plds_set_update(plds_set_t *s, const int32_t *edges, const int64_t *offsets) {
    if (!s || !offsets) return set_status(PLDS_EINVAL);
    const int32_t G = s->count;
    const int64_t total = offsets[2 * G];
    if (offsets[0] != 0 || total < 0 || (total > 0 && !edges)) return set_status(PLDS_EINVAL);
    for (int32_t k = 0; k < 2 * G; ++k)
        if (offsets[k + 1] < offsets[k]) return set_status(PLDS_EINVAL);
    for (plds *h : s->g) {
        if (h->poisoned) return set_status(PLDS_EPOISONED);
        h->orient_ok = false;
    }
    plds *o = s->owner;
    cudaSetDevice(o->device);
    const int32_t *dedges = edges;
    if (total > 0 && !is_device_ptr(edges)) {
        if (total > s->edges_cap) {
            if (!dev_get(o, s->edges, sizeof(int32_t) * 2 * (size_t)total)) return set_status(PLDS_ENOMEM);
            s->edges_cap = total;
        }
        cudaMemcpyAsync(s->edges.p, edges, sizeof(int32_t) * 2 * (size_t)total, cudaMemcpyHostToDevice, s->stream);
        dedges = P<int32_t>(s->edges);
    }
    // graphs still to run this round (all at first; then the ones that needed a bigger pool)
    std::vector<int32_t> todo(s->order);
    Ctl *dctl = P<Ctl>(s->ctls);
    for (int attempt = 0; attempt < 4 && !todo.empty(); ++attempt) {
        const int32_t m = (int32_t)todo.size();
        for (int32_t j = 0; j < m; ++j) {
            const int32_t gi = todo[j];
            plds *h = s->g[gi];
            const int64_t bi = offsets[2 * gi + 1] - offsets[2 * gi], bd = offsets[2 * gi + 2] - offsets[2 * gi + 1];
            if (!ensure_batch_scratch(h, std::max<int64_t>(std::max(bi, bd), 1))) return set_status(PLDS_ENOMEM);
            std::memset(&h->last, 0, sizeof(h->last));
            h->last.submitted = bi + bd;
            for (int half = 0; half < 2; ++half) {
                const int64_t b = half == 0 ? bi : bd;
                if ((int64_t)h->stamp_base + 2 * (int64_t)h->T.K + 8 >= 0x7fffffff) {
                    cudaMemsetAsync(h->stamp.p, 0, sizeof(int32_t) * (size_t)h->n, s->stream);
                    h->stamp_base = 1;
                }
                GraphCtx g = make_ctx(h, half == 0 ? kOpInsert : kOpDelete, dedges + 2 * offsets[2 * gi + half], b);
                g.ctl = dctl + 2 * j + half;
                g.trace = nullptr;
                g.trace_cap = 0;
                s->h_items[j].half[half] = g;
                if (b > 0) h->stamp_base += h->T.K + 2;
            }
        }
        // the first pass over all graphs replays the captured round; reruns launch directly
        if (cudaStreamSynchronize(s->stream) != cudaSuccess || set_launch(s, m, attempt == 0) != 0 ||
            cudaStreamSynchronize(s->run) != cudaSuccess) {
            cudaGetLastError();
            for (plds *h : s->g) h->poisoned = true;
            return set_status(PLDS_EDEVICE);
        }
        o->launches += 1;
        std::vector<int32_t> again;
        for (int32_t j = 0; j < m; ++j) {
            const int32_t gi = todo[j];
            plds *h = s->g[gi];
            const Ctl &ci = s->h_ctls[2 * j], &cd = s->h_ctls[2 * j + 1];
            // the deletion half runs only after a clean insertion half
            const int32_t err = ci.err ? ci.err : cd.err;
            if (err & kErrInvalidId) return set_status(PLDS_EINVAL);
            if (err == kErrNeedPool) {
                int rc = grow_pool(h, (int64_t)ci.grow_total);
                if (rc) return set_status(rc);
                again.push_back(gi);
                continue;
            }
            if (err) {
                h->poisoned = true;
                h->last.err_bits = err;
                h->last.err_site = ci.err ? ci.err_site : cd.err_site;
                return set_status(PLDS_EINTERNAL);
            }
            for (const Ctl *c : {&ci, &cd}) {
                h->last.self_loops += (int64_t)c->st[kStSelfLoops];
                h->last.filtered += (int64_t)c->st[kStFiltered];
                h->last.valid += (int64_t)c->vcount;
                h->last.rounds += (int64_t)c->st[kStRounds];
                h->last.moves += (int64_t)c->st[kStMoves];
                h->last.visits += (int64_t)c->st[kStVisits];
                h->last.dl_evals += (int64_t)c->st[kStDlEvals];
                h->last.dl_visits += (int64_t)c->st[kStDlVisits];
                h->last.slots_scanned += (int64_t)c->st[kStSlotsScanned];
                h->last.up_visits += (int64_t)c->st[kStUpVisits];
                h->last.affected += (int64_t)c->st[kStAffected];
                h->last.skipped_rounds += (int64_t)c->st[kStSkipRounds];
                h->last.skipped_moves += (int64_t)c->st[kStSkipMoves];
                h->last.skipped_visits += (int64_t)c->st[kStSkipVisits];
                h->last.skipped_up_visits += (int64_t)c->st[kStSkipUpVisits];
            }
            const int64_t bi = offsets[2 * gi + 1] - offsets[2 * gi], bd = offsets[2 * gi + 2] - offsets[2 * gi + 1];
            h->last.duplicates = (bi > 0 ? bi - (int64_t)ci.st[kStSelfLoops] - (int64_t)ci.ucount : 0) +
                                 (bd > 0 ? bd - (int64_t)cd.st[kStSelfLoops] - (int64_t)cd.ucount : 0);
        }
        todo.swap(again);
    }
    return set_status(todo.empty() ? PLDS_OK : PLDS_ENOMEM);
}

extern "C" int plds_set_tune(plds_set_t *s, const plds_tuning *t) {
    if (!s || !t) return set_status(PLDS_EINVAL);
    for (plds *h : s->g) {
        plds_tuning x = h->tune;
        x.thread_max_cap = t->thread_max_cap;
        x.block_cap = t->block_cap;
        x.load_num = t->load_num;
        x.load_den = t->load_den;
        x.list_cap = t->list_cap;
        const int rc = plds_set_tuning(h, &x);
        if (rc) return rc;
    }
    return set_status(PLDS_OK);
}

// ---------------------------------------------------------------------------
// Autotuner: coordinate descent over the knobs that change only speed.
// ---------------------------------------------------------------------------
namespace {
constexpr int32_t kTuneThread[] = {4, 8, 16, 32, 64};
constexpr int32_t kTuneBlock[] = {1024, 2048, 4096, 8192, 16384};
constexpr int32_t kTuneLoad[][2] = {{1, 2}, {5, 8}, {3, 4}, {7, 8}};
constexpr int32_t kTuneList[] = {128, 256, 1024, 1 << 30};

bool same_knobs(const plds_tuning &a, const plds_tuning &b) {
    return a.thread_max_cap == b.thread_max_cap && a.block_cap == b.block_cap && a.load_num == b.load_num &&
           a.load_den == b.load_den && a.list_cap == b.list_cap;
}

struct SetTuneCtx {
    plds_set *s;
    int32_t rounds;
    const int32_t *const *edges;
    const int64_t *const *offsets;
    int32_t timed_from;
    int status;
};

// One evaluation: a scratch set of the same graph sizes, the sample rounds, the
// wall time of the timed ones (every plds_set_update call returns when done).
double set_trial_cost(const plds_tuning *t, void *vctx) {
    SetTuneCtx *c = static_cast<SetTuneCtx *>(vctx);
    plds_set *s = c->s;
    plds_set_t *x = plds_set_create(s->count, s->ns.data(), s->delta, s->lambda, s->has_alloc ? &s->alloc : nullptr,
                                    (void *)s->stream);
    if (!x) {
        c->status = plds_last_status();
        return -1.0;
    }
    int rc = plds_set_tune(x, t);
    double secs = 0.0;
    for (int32_t r = 0; r < c->rounds && rc == PLDS_OK; ++r) {
        const auto t0 = std::chrono::steady_clock::now();
        rc = plds_set_update(x, c->edges[r], c->offsets[r]);
        if (r >= c->timed_from) secs += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    plds_set_destroy(x);
    if (rc != PLDS_OK) {
        c->status = rc;
        return -1.0;
    }
    return secs;
}
}  // namespace

extern "C" int plds_tune_search(const plds_tuning *start, plds_tune_cost cost, void *ctx, int32_t max_trials,
                                plds_tuning *best) {
    if (!start || !cost || !best || max_trials < 1) return set_status(PLDS_EINVAL);
    plds_tuning cur = *start;
    if (cur.thread_max_cap <= 0) cur.thread_max_cap = 16;
    if (cur.block_cap <= 0) cur.block_cap = 4096;
    if (cur.load_num <= 0 || cur.load_den <= 0) {
        cur.load_num = 3;
        cur.load_den = 4;
    }
    if (cur.list_cap <= 0) cur.list_cap = 256;
    std::vector<std::pair<plds_tuning, double>> seen;  // every evaluation, to skip repeats
    int32_t trials = 0;
    // 0: cost in *c; 1: budget spent; -1: the cost function gave up
    auto eval = [&](const plds_tuning &t, double *c) -> int {
        for (const auto &e : seen)
            if (same_knobs(e.first, t)) {
                *c = e.second;
                return 0;
            }
        if (trials >= max_trials) return 1;
        const double v = cost(&t, ctx);
        ++trials;
        if (!(v >= 0.0)) return -1;
        seen.push_back({t, v});
        *c = v;
        return 0;
    };
    double cur_cost = 0.0;
    if (eval(cur, &cur_cost) < 0) return set_status(PLDS_EINTERNAL);
    bool improved = true, spent = false;
    while (improved && !spent) {
        improved = false;
        for (int knob = 0; knob < 4 && !spent; ++knob) {
            const int nv = knob >= 2 ? 4 : 5;
            for (int v = 0; v < nv; ++v) {
                plds_tuning t = cur;
                if (knob == 0) {
                    t.thread_max_cap = kTuneThread[v];
                } else if (knob == 1) {
                    t.block_cap = kTuneBlock[v];
                } else if (knob == 2) {
                    t.load_num = kTuneLoad[v][0];
                    t.load_den = kTuneLoad[v][1];
                } else {
                    t.list_cap = kTuneList[v];
                }
                if (same_knobs(t, cur)) continue;
                double c = 0.0;
                const int rc = eval(t, &c);
                if (rc < 0) return set_status(PLDS_EINTERNAL);
                if (rc > 0) {
                    spent = true;
                    break;
                }
                if (c < 0.98 * cur_cost) {
                    cur = t;
                    cur_cost = c;
                    improved = true;
                }
            }
        }
    }
    *best = cur;
    set_status(PLDS_OK);
    return trials;
}

extern "C" int plds_set_autotune(plds_set_t *s, int32_t rounds, const int32_t *const *edges,
                                 const int64_t *const *offsets, int32_t timed_from, int32_t max_trials,
                                 plds_tuning *best) {
    if (!s || rounds < 1 || !edges || !offsets || timed_from < 0 || timed_from >= rounds || max_trials < 1)
        return set_status(PLDS_EINVAL);
    SetTuneCtx c{s, rounds, edges, offsets, timed_from, PLDS_OK};
    plds_tuning out{};
    const int trials = plds_tune_search(&s->g[0]->tune, set_trial_cost, &c, max_trials, &out);
    if (trials < 0) return set_status(c.status != PLDS_OK ? c.status : trials);
    const int rc = plds_set_tune(s, &out);
    if (rc) return rc;
    if (best) *best = out;
    return set_status(PLDS_OK);
}

namespace {
struct HandleTuneCtx {
    plds *h;
    const int32_t *edges;
    const int64_t *offsets;
    const int32_t *kinds;
    int32_t nbatches, timed_from;
    int status;
};

// One evaluation: a scratch handle configured like the handle being tuned, the
// sample batches applied to it, the wall time of the timed ones (each call is
// synchronous).
double handle_trial_cost(const plds_tuning *t, void *ctx) {
    auto *c = static_cast<HandleTuneCtx *>(ctx);
    plds *h = c->h;
    plds *x = plds_create_ex(h->n, h->delta, h->lambda, h->levels_per_group, h->custom_alloc ? &h->alloc : nullptr,
                             (void *)h->stream, h->flags);
    if (!x) {
        c->status = plds_last_status();
        return -1.0;
    }
    plds_tuning tt = h->tune;
    tt.thread_max_cap = t->thread_max_cap;
    tt.block_cap = t->block_cap;
    tt.load_num = t->load_num;
    tt.load_den = t->load_den;
    tt.list_cap = t->list_cap;
    tt.trace_rounds = 0;
    tt.track_orientation = 0;
    int rc = plds_set_tuning(x, &tt);
    double secs = 0.0;
    for (int32_t b = 0; b < c->nbatches && rc == PLDS_OK; ++b) {
        const int32_t *e = c->edges + 2 * c->offsets[b];
        const int64_t B = c->offsets[b + 1] - c->offsets[b];
        const auto t0 = std::chrono::steady_clock::now();
        rc = c->kinds[b] ? plds_batch_delete(x, e, B) : plds_batch_insert(x, e, B);
        if (b >= c->timed_from) secs += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    plds_destroy(x);
    if (rc != PLDS_OK) {
        c->status = rc;
        return -1.0;
    }
    return secs;
}
}  // namespace

extern "C" int plds_autotune(plds_t *h, const int32_t *edges, const int64_t *offsets, const int32_t *kinds,
                             int32_t nbatches, int32_t timed_from, int32_t max_trials, plds_tuning *best) {
    if (!h || !edges || !offsets || !kinds || nbatches < 1 || timed_from < 0 || timed_from >= nbatches ||
        max_trials < 1)
        return set_status(PLDS_EINVAL);
    if (h->poisoned) return set_status(PLDS_EPOISONED);
    for (int32_t b = 0; b < nbatches; ++b)
        if (offsets[b] < 0 || offsets[b + 1] < offsets[b] || (kinds[b] != 0 && kinds[b] != 1))
            return set_status(PLDS_EINVAL);
    HandleTuneCtx c{h, edges, offsets, kinds, nbatches, timed_from, PLDS_OK};
    plds_tuning out{};
    const int trials = plds_tune_search(&h->tune, handle_trial_cost, &c, max_trials, &out);
    if (trials < 0) return set_status(c.status != PLDS_OK ? c.status : trials);
    h->tune.thread_max_cap = out.thread_max_cap;
    h->tune.block_cap = out.block_cap;
    h->tune.load_num = out.load_num;
    h->tune.load_den = out.load_den;
    h->tune.list_cap = out.list_cap;
    if (best) *best = h->tune;
    return set_status(PLDS_OK);
}

extern "C" void plds_set_destroy(plds_set_t *s) {
    if (!s) return;
    if (s->exec) cudaGraphExecDestroy(s->exec);
    if (s->graph) cudaGraphDestroy(s->graph);
    if (s->run) {
        cudaStreamSynchronize(s->run);
        cudaStreamDestroy(s->run);
    }
    if (s->owner) {
        dev_free(s->owner, s->items);
        dev_free(s->owner, s->ctls);
        dev_free(s->owner, s->next);
        dev_free(s->owner, s->edges);
        cudaStreamSynchronize(s->stream);
    }
    if (s->h_items) cudaFreeHost(s->h_items);
    if (s->h_ctls) cudaFreeHost(s->h_ctls);
    for (plds *h : s->g) plds_destroy(h);
    cudaGetLastError();
    delete s;
}

// ---------------------------------------------------------------------------
// Serving form: a device-resident request loop.
//
// One persistent cooperative kernel serves a graph.  Requests (an insertion
// batch, a deletion batch, or a coreness query) sit in a ring of slots in
// pinned host memory that the device reads directly; the kernel's leader thread
// polls the next slot, the grid applies the request with the same routines as a
// single batch call, and the leader writes the completion record back into the
// slot.  Requests are applied in submission order.  The host admits a new
// request whenever a slot is free and the adjacency could grow to hold it: its
// copy-in overlaps with the device working on earlier requests, and no kernel
// launch or host synchronisation sits between requests.
//
// Continuous batching: when the leader finds several consecutive update
// requests of the same kind already waiting, it applies them as ONE batch (up
// to merge_cap edges, at most kMaxSeg requests): the grid gathers their edges
// into one device buffer, validating ids per request so that a request with an
// id out of range is rejected alone.  Every merged request's completion names
// the first ticket and the number of requests of the batch it went into, so the
// schedule can be replayed batch by batch.  With merge_cap 0 every request is
// its own batch (unchanged boundaries).  Queries are never merged: they see the
// state after every earlier request.
//
// The loop exits after an idle period or when the adjacency pool needs to grow
// (the host grows it, gated by free HBM, and relaunches).
// ---------------------------------------------------------------------------
namespace {
enum : int32_t { kSlotFree = 0, kSlotReady = 1, kSlotDone = 2 };
enum : int32_t { kReqInsert = 0, kReqDelete = 1, kReqCoreness = 2 };
enum : int32_t { kExitNone = 0, kExitIdle = 1, kExitNeedPool = 2, kExitError = 3 };
constexpr int kMaxSeg = 64;  // requests merged into one batch at most

struct alignas(64) ReqSlot {
    int32_t state;  // kSlot*
    int32_t op;     // kReq*
    int64_t B;
    const int32_t *edges;  // device-accessible
    double *out;           // device-accessible (coreness queries)
    int64_t ticket;
    int64_t merge_cap;  // edges one merged batch may hold (0: never merge)
    // written by the device
    int32_t status;   // device error bits
    int32_t batch_n;  // requests in the batch this one was applied in
    int64_t batch_first;  // ticket of that batch's first request
    uint64_t t_begin, t_end;  // device globaltimer
    unsigned long long pool_top;  // adjacency slots handed out after the request
    unsigned long long st[kStCount];
    unsigned long long valid;
};

struct ServeCtl {  // device memory
    int32_t exit_reason;
    int32_t cmd;
    int64_t head;        // next slot sequence number
    int32_t stamp_next;  // stamps of the next request start here
    int32_t nseg;        // requests in the current batch (0: a query or an unmerged request)
    unsigned long long grow_total;
    int64_t seg_total;   // edges gathered (after rejected requests are dropped)
    ReqSlot cur;         // the head request (copied from the ring)
    const int2 *seg_ptr[kMaxSeg];
    int64_t seg_off[kMaxSeg + 1];
    int32_t seg_bad[kMaxSeg];
};

struct ServeArgs {
    ReqSlot *ring;  // device pointer of the pinned ring
    int32_t slots;
    int64_t idle_ns;
    ServeCtl *sc;
    const double *powtab;
    int2 *ebuf;  // gathered edges of a merged batch [max_batch]
};
}  // namespace

// Word-by-word copy that reads through volatile loads (the source may be host memory
// the host is writing, or device memory written by another block).
__device__ __forceinline__ void copy_slot(ReqSlot *dst, const ReqSlot *src) {
    const volatile int32_t *sv = reinterpret_cast<const volatile int32_t *>(src);
    int32_t *dv = reinterpret_cast<int32_t *>(dst);
    for (int k = 0; k < (int)(sizeof(ReqSlot) / 4); ++k) dv[k] = sv[k];
}

// Leader: extend the batch that starts with the head request by the waiting
// requests that follow it (same kind, total edges within the cap).
__device__ void serve_select(const ServeArgs &a, ServeCtl *sc) {
    const ReqSlot &c = sc->cur;
    sc->nseg = 0;
    if (c.op == kReqCoreness || c.merge_cap <= 0 || c.B > c.merge_cap) return;
    int64_t total = c.B;
    sc->seg_ptr[0] = reinterpret_cast<const int2 *>(c.edges);
    sc->seg_off[0] = 0;
    sc->seg_bad[0] = 0;
    int ns = 1;
    for (int j = 1; j < a.slots && ns < kMaxSeg; ++j) {
        const ReqSlot *r = a.ring + ((sc->head + j) % a.slots);
        if (*(volatile const int32_t *)&r->state != kSlotReady) break;
        __threadfence_system();
        const int32_t op = *(volatile const int32_t *)&r->op;
        const int64_t B = *(volatile const int64_t *)&r->B;
        if (op != c.op || total + B > c.merge_cap) break;
        sc->seg_ptr[ns] = reinterpret_cast<const int2 *>(*(const int32_t *volatile *)&r->edges);
        sc->seg_off[ns] = total;
        sc->seg_bad[ns] = 0;
        total += B;
        ++ns;
    }
    sc->seg_off[ns] = total;
    sc->seg_total = total;
    sc->nseg = ns > 1 ? ns : 0;  // a request alone is read in place
}

// Grid: copy the batch's requests into one contiguous edge array; with `check`,
// flag each request holding an id outside [0, n).  Segment offsets are in shared
// memory (s_off[0..ns]).
__device__ void serve_gather(GridTeam &T, const ServeCtl *sc, int ns, const int64_t *s_off, int2 *ebuf, int32_t n,
                             bool check, int32_t *bad) {
    const int64_t total = s_off[ns];
    for (int64_t i = T.tid(); i < total; i += T.nthreads()) {
        int lo = 0, hi = ns - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const int2 uv = sc->seg_ptr[lo][i - s_off[lo]];
        if (check && (uv.x < 0 || uv.x >= n || uv.y < 0 || uv.y >= n)) *(volatile int32_t *)&bad[lo] = 1;
        ebuf[i] = uv;
    }
}

__global__ void __launch_bounds__(512) k_serve(const __grid_constant__ GraphCtx base, const ServeArgs a) {
    extern __shared__ int32_t sh[];
    __shared__ int64_t s_off[kMaxSeg + 1];
    GridTeam T{base.ctl, base.wait_limit_ns, base.barrier_sleep_ns};
    ServeCtl *sc = a.sc;
    for (;;) {
        // the leader waits for the next slot (bounded by the idle limit)
        if (T.leader()) {
            ReqSlot *r = a.ring + (sc->head % a.slots);
            const uint64_t t0 = global_ns();
            int32_t st;
            while ((st = *(volatile int32_t *)&r->state) != kSlotReady && global_ns() - t0 < (uint64_t)a.idle_ns)
                __nanosleep(256);
            if (st == kSlotReady) {
                __threadfence_system();
                copy_slot(&sc->cur, r);
                serve_select(a, sc);
                sc->cmd = 1;
            } else {
                sc->cmd = 0;
                sc->exit_reason = kExitIdle;
            }
            __threadfence();
        }
        if (!T.sync()) return;
        if (ld_volatile(&sc->cmd) == 0) return;
        // a fresh control block and key set for this request (the barrier words stay)
        {
            int32_t *cw = reinterpret_cast<int32_t *>(base.ctl);
            const int first = (int)(offsetof(Ctl, err) / 4);
            for (int k = T.tid() + first; k < (int)(sizeof(Ctl) / 4); k += T.nthreads()) cw[k] = 0;
            for (int64_t k = T.tid(); k < base.hcap; k += T.nthreads()) base.hset[k] = kEmptyKey;
            for (int k = T.tid(); k <= base.K; k += T.nthreads()) base.bins[k] = 0;
            if (sc->stamp_next + 2 * base.K + 8 >= 0x7fffffff) {  // stamps wrap: clear them
                for (int k = T.tid(); k < base.n; k += T.nthreads()) base.stamp[k] = 0;
            }
        }
        ReqSlot req;
        copy_slot(&req, &sc->cur);
        const int ns = ld_volatile(&sc->nseg);
        if (ns > 0) {  // gather the batch's requests, rejecting those with a bad id
            for (int k = threadIdx.x; k <= ns; k += blockDim.x) s_off[k] = sc->seg_off[k];
            __syncthreads();
            serve_gather(T, sc, ns, s_off, a.ebuf, base.n, true, sc->seg_bad);
            if (!T.sync()) return;
            bool anybad = false;
            for (int k = 0; k < ns; ++k) anybad |= ld_volatile(&sc->seg_bad[k]) != 0;
            if (anybad) {  // gather again without the rejected requests (they keep length 0)
                __syncthreads();
                if (threadIdx.x == 0) {
                    int64_t t = 0;
                    for (int k = 0; k < ns; ++k) {
                        s_off[k] = t;
                        if (!ld_volatile(&sc->seg_bad[k])) t += sc->seg_off[k + 1] - sc->seg_off[k];
                    }
                    s_off[ns] = t;
                }
                __syncthreads();
                if (T.leader()) sc->seg_total = s_off[ns];
                // a zero-length segment is never selected by the search below (offsets
                // equal), so the remaining requests' edges land contiguously
                serve_gather(T, sc, ns, s_off, a.ebuf, base.n, false, sc->seg_bad);
            }
        }
        if (!T.sync()) return;
        int32_t sbase = sc->stamp_next;
        if (sbase + 2 * base.K + 8 >= 0x7fffffff) sbase = 1;
        const uint64_t t_begin = global_ns();
        if (req.op == kReqCoreness) {
            for (int64_t v = T.tid(); v < base.n; v += T.nthreads()) {
                int32_t g = -1;
                if (base.deg[v] > 0) g = max((base.level[v] + 1) / base.Lg - 1, 0);
                req.out[v] = g < 0 ? 0.0 : a.powtab[g];
            }
        } else {
            const BatchIn in{ns > 0 ? reinterpret_cast<const int32_t *>(a.ebuf) : req.edges,
                             ns > 0 ? *(volatile const int64_t *)&sc->seg_total : req.B,
                             req.op == kReqInsert ? kOpInsert : kOpDelete, sbase};
            run_batch(T, base, in, sh, 0);
        }
        const bool ok = T.sync();
        if (T.leader()) {
            const int32_t err = ld_volatile(&base.ctl->err);
            if (err == kErrNeedPool) {  // leave the slots ready; the host grows the pool and relaunches
                sc->exit_reason = kExitNeedPool;
                sc->grow_total = base.ctl->grow_total;
                sc->stamp_next = sbase + base.K + 2;
            } else {
                const int nr = ns > 0 ? ns : 1;
                const uint64_t t_end = global_ns();
                const unsigned long long top = *(volatile unsigned long long *)base.pool_top;
                for (int j = 0; j < nr; ++j) {
                    ReqSlot *r = a.ring + ((sc->head + j) % a.slots);
                    r->status = (ns > 0 && ld_volatile(&sc->seg_bad[j])) ? kErrInvalidId : err;
                    r->batch_n = nr;
                    r->batch_first = req.ticket;
                    r->t_begin = t_begin;
                    r->t_end = t_end;
                    r->pool_top = top;
                    for (int k = 0; k < kStCount; ++k) r->st[k] = base.ctl->st[k];
                    r->valid = base.ctl->vcount;
                }
                __threadfence_system();
                for (int j = 0; j < nr; ++j)
                    *(volatile int32_t *)&a.ring[(sc->head + j) % a.slots].state = kSlotDone;
                sc->head += nr;
                sc->stamp_next = sbase + base.K + 2;
                if (err) sc->exit_reason = kExitError;
            }
            __threadfence();
        }
        if (!ok) return;
        if (!T.sync()) return;
    }
}

struct plds_server {
    plds *h = nullptr;
    int32_t slots = 0;
    int64_t max_batch = 0;
    ReqSlot *ring = nullptr;  // pinned, mapped
    ReqSlot *ring_dev = nullptr;
    std::vector<int32_t *> stage;  // pinned, mapped edge staging per slot
    std::vector<int32_t *> stage_dev;
    std::vector<int64_t> stage_cap;  // edges; allocated on first use by a pageable input
    double *qbuf = nullptr;  // pinned, mapped coreness staging
    double *qbuf_dev = nullptr;
    std::vector<double *> qdest;  // where a finished query's values go (when staged)
    DevBuf sc, ebuf;
    cudaStream_t run = nullptr;
    cudaEvent_t done = nullptr;
    bool running = false;
    int64_t next_seq = 0;  // sequence number of the next submitted request
    int64_t done_seq = 0;  // all sequence numbers below have been collected
    int64_t idle_ns = 20ll * 1000 * 1000;
    int64_t merge_cap = 0;        // edges per merged batch (0: unchanged boundaries)
    int64_t pool_limit = 0;       // bytes the adjacency pool may take (0: free HBM only)
    int64_t pool_used = 0;        // adjacency slots handed out, as last reported
    int64_t inflight_need = 0;    // worst-case slots of admitted, unfinished insertions
    std::vector<int64_t> need;    // per ring slot
    std::vector<plds_request_result> finished;
};

static int64_t now_monotonic_ns() {
    timespec ts{};
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

// Worst-case adjacency slots an insertion batch of B edges can take: both endpoint
// tables may double, at load num/den.
static int64_t insert_need_slots(const plds *h, int64_t B) {
    const int64_t num = h->tune.load_num > 0 ? h->tune.load_num : 3;
    const int64_t den = h->tune.load_den > 0 ? h->tune.load_den : 4;
    return (4 * B * den + num - 1) / num;
}

static int server_launch(plds_server *sv) {
    plds *h = sv->h;
    const int threads = block_threads(h);
    const size_t smem = smem_bytes(threads);
    static std::atomic<bool> attr_serve[kAttrDevices];
    raise_smem_limit(k_serve, attr_serve, h->device);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_serve, threads, smem);
    const int per_sm = h->tune.blocks_per_sm > 0 ? std::min(h->tune.blocks_per_sm, occ) : 1;
    if (per_sm < 1) return PLDS_EDEVICE;
    GraphCtx g = make_ctx(h, kOpInsert, nullptr, 0);
    g.trace = nullptr;
    g.trace_cap = 0;
    // A loop that stopped on an error may have left grid-barrier arrivals counted
    // (blocks leave a barrier early once the error word is set): start clean.
    cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), sv->run);
    cudaMemsetAsync(&P<ServeCtl>(sv->sc)->exit_reason, 0, sizeof(int32_t) * 2, sv->run);
    ServeArgs a{sv->ring_dev, sv->slots, sv->idle_ns, P<ServeCtl>(sv->sc), P<double>(h->powtab), P<int2>(sv->ebuf)};
    void *args[] = {(void *)&g, (void *)&a};
    if (cudaLaunchCooperativeKernel((const void *)k_serve, dim3(h->num_sms * per_sm), dim3(threads), args, smem,
                                    sv->run) != cudaSuccess) {
        cudaGetLastError();
        return PLDS_EDEVICE;
    }
    cudaEventRecord(sv->done, sv->run);
    h->launches++;
    sv->running = true;
    return PLDS_OK;
}

// If the loop has stopped: read why, grow the pool if asked, relaunch when
// requests are waiting.  Returns a status.
static int server_service(plds_server *sv) {
    if (!sv->running) return PLDS_OK;
    if (cudaEventQuery(sv->done) == cudaErrorNotReady) return PLDS_OK;
    cudaGetLastError();
    sv->running = false;
    plds *h = sv->h;
    ServeCtl c{};
    if (cudaMemcpy(&c, sv->sc.p, sizeof(ServeCtl), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        h->poisoned = true;
        return PLDS_EDEVICE;
    }
    h->stamp_base = c.stamp_next;
    Ctl hc{};
    cudaMemcpy(&hc, h->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost);
    if (hc.err & kErrTimeout) {
        h->poisoned = true;
        return PLDS_ETIMEOUT;
    }
    int32_t reset = kExitNone;
    cudaMemcpy(&reinterpret_cast<ServeCtl *>(sv->sc.p)->exit_reason, &reset, 4, cudaMemcpyHostToDevice);
    if (c.exit_reason == kExitNeedPool) {
        const int64_t saved = h->pool_limit;
        h->pool_limit = sv->pool_limit;
        int rc = grow_pool(h, (int64_t)c.grow_total);
        h->pool_limit = saved;
        if (rc) return rc;
        cudaDeviceSynchronize();
        sv->pool_used = h->pool_live;
    }
    if (sv->next_seq > c.head) return server_launch(sv);  // requests are waiting
    return PLDS_OK;
}

// Move finished requests out of the ring; frees their slots.
static void server_collect(plds_server *sv) {
    while (sv->done_seq < sv->next_seq) {
        ReqSlot *r = sv->ring + (sv->done_seq % sv->slots);
        if (*(volatile int32_t *)&r->state != kSlotDone) break;
        std::atomic_thread_fence(std::memory_order_acquire);
        plds_request_result out{};
        out.ticket = r->ticket;
        out.op = r->op;
        out.status = r->status == 0 ? PLDS_OK : ((r->status & kErrInvalidId) ? PLDS_EINVAL : PLDS_EINTERNAL);
        out.valid = (int64_t)r->valid;
        out.rounds = (int64_t)r->st[kStRounds];
        out.moves = (int64_t)r->st[kStMoves];
        out.device_ns = (int64_t)(r->t_end - r->t_begin);
        out.batch_first = r->batch_first;
        out.batch_size = r->batch_n;
        out.done_ns = now_monotonic_ns();
        const int slot = (int)(sv->done_seq % sv->slots);
        sv->pool_used = (int64_t)r->pool_top;
        sv->inflight_need -= sv->need[slot];
        sv->need[slot] = 0;
        if (r->op == kReqCoreness && sv->qdest[slot]) {
            std::memcpy(sv->qdest[slot], sv->qbuf, sizeof(double) * (size_t)sv->h->n);
            sv->qdest[slot] = nullptr;
        }
        sv->finished.push_back(out);
        *(volatile int32_t *)&r->state = kSlotFree;
        sv->done_seq++;
    }
}

static void server_free(plds_server *sv) {
    if (sv->run) {
        cudaStreamSynchronize(sv->run);
        cudaStreamDestroy(sv->run);
    }
    if (sv->done) cudaEventDestroy(sv->done);
    if (sv->ring) cudaFreeHost(sv->ring);
    for (int32_t *p : sv->stage)
        if (p) cudaFreeHost(p);
    if (sv->qbuf) cudaFreeHost(sv->qbuf);
    if (sv->h) {
        dev_free(sv->h, sv->sc);
        dev_free(sv->h, sv->ebuf);
    }
    cudaGetLastError();
    delete sv;
}

extern "C" plds_server_t *plds_server_create(plds_t *h, int32_t slots, int64_t max_batch) {
    if (!h || slots < 1 || slots > 4096 || max_batch < 1) {
        set_status(PLDS_EINVAL);
        return nullptr;
    }
    if (h->poisoned) {
        set_status(PLDS_EPOISONED);
        return nullptr;
    }
    plds_server *sv = new (std::nothrow) plds_server();
    if (!sv) {
        set_status(PLDS_ENOMEM);
        return nullptr;
    }
    sv->h = h;
    sv->slots = slots;
    sv->max_batch = max_batch;
    cudaSetDevice(h->device);
    bool ok = ensure_batch_scratch(h, max_batch) && dev_get(h, sv->sc, sizeof(ServeCtl)) &&
              dev_get(h, sv->ebuf, sizeof(int2) * (size_t)max_batch) &&
              cudaStreamCreateWithFlags(&sv->run, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&sv->done, cudaEventDisableTiming) == cudaSuccess &&
              cudaHostAlloc((void **)&sv->ring, sizeof(ReqSlot) * slots, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&sv->ring_dev, sv->ring, 0) == cudaSuccess &&
              cudaHostAlloc((void **)&sv->qbuf, sizeof(double) * (size_t)h->n, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer((void **)&sv->qbuf_dev, sv->qbuf, 0) == cudaSuccess;
    if (ok) {
        std::memset(sv->ring, 0, sizeof(ReqSlot) * slots);
        sv->stage.assign(slots, nullptr);
        sv->stage_dev.assign(slots, nullptr);
        sv->qdest.assign(slots, nullptr);
        sv->need.assign(slots, 0);
        sv->merge_cap = max_batch;
        sv->pool_used = h->pool_cap;  // unknown until the first completion: assume full
        sv->stage_cap.assign(slots, 0);
    }
    if (ok) {
        ServeCtl c{};
        c.stamp_next = h->stamp_base;
        cudaStreamSynchronize(h->stream);
        ok = cudaMemcpy(sv->sc.p, &c, sizeof(ServeCtl), cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(h->ctl.p, 0, sizeof(Ctl)) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        server_free(sv);
        set_status(PLDS_ENOMEM);
        return nullptr;
    }
    set_status(PLDS_OK);
    return sv;
}

extern "C" int plds_server_submit(plds_server_t *sv, int32_t op, const int32_t *edges, int64_t B, double *out,
                                  int64_t *ticket) {
    if (!sv || op < kReqInsert || op > kReqCoreness) return set_status(PLDS_EINVAL);
    if (op != kReqCoreness && (B < 0 || B > sv->max_batch || (B > 0 && !edges))) return set_status(PLDS_EINVAL);
    if (op == kReqCoreness && !out) return set_status(PLDS_EINVAL);
    plds *h = sv->h;
    if (h->poisoned) return set_status(PLDS_EPOISONED);
    h->orient_ok = false;
    cudaSetDevice(h->device);
    // wait for a free slot (collect finished requests, keep the loop alive)
    const auto t0 = std::chrono::steady_clock::now();
    while (sv->next_seq - sv->done_seq >= sv->slots) {
        server_collect(sv);
        int rc = server_service(sv);
        if (rc) return set_status(rc);
        if (std::chrono::steady_clock::now() - t0 > std::chrono::nanoseconds(h->wait_limit_ns))
            return set_status(PLDS_ETIMEOUT);
    }
    // admission: the adjacency must be able to grow to hold the batch (worst case)
    const int64_t need = op == kReqInsert ? insert_need_slots(h, B) : 0;
    for (;;) {
        int64_t free_b = 0;
        if (need > 0 && h->pool_cap - sv->pool_used - sv->inflight_need < need) {
            size_t fb = 0, tb = 0;
            if (cudaMemGetInfo(&fb, &tb) != cudaSuccess) {
                cudaGetLastError();
                fb = 0;
            }
            free_b = std::max<int64_t>(0, (int64_t)fb - kHbmReserve);
            if (sv->pool_limit > 0) free_b = std::min<int64_t>(free_b, sv->pool_limit);
        }
        const int d = plds_server_admission(h->pool_cap, sv->pool_used, sv->inflight_need, need, free_b);
        if (d == 0) break;
        if (d != 1) return set_status(PLDS_ENOMEM);
        server_collect(sv);
        int rc = server_service(sv);
        if (rc) return set_status(rc);
        if (std::chrono::steady_clock::now() - t0 > std::chrono::nanoseconds(h->wait_limit_ns))
            return set_status(PLDS_ETIMEOUT);
    }
    bool out_dev = false;
    void *out_devptr = nullptr;
    if (op == kReqCoreness) {
        cudaPointerAttributes pa{};
        out_dev = cudaPointerGetAttributes(&pa, out) == cudaSuccess && pa.devicePointer &&
                  (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged || pa.type == cudaMemoryTypeHost);
        out_devptr = pa.devicePointer;
        cudaGetLastError();
        // pageable output goes through the one staging buffer: one such query at a time
        while (!out_dev && std::any_of(sv->qdest.begin(), sv->qdest.end(), [](double *d) { return d != nullptr; })) {
            server_collect(sv);
            int rc = server_service(sv);
            if (rc) return set_status(rc);
            if (std::chrono::steady_clock::now() - t0 > std::chrono::nanoseconds(h->wait_limit_ns))
                return set_status(PLDS_ETIMEOUT);
        }
    }
    const int slot = (int)(sv->next_seq % sv->slots);
    ReqSlot *r = sv->ring + slot;
    r->op = op;
    r->B = op == kReqCoreness ? 0 : B;
    r->ticket = sv->next_seq;
    r->merge_cap = sv->merge_cap;
    r->edges = nullptr;
    r->out = nullptr;
    if (op != kReqCoreness && B > 0) {
        cudaPointerAttributes pa{};
        const bool dev = cudaPointerGetAttributes(&pa, edges) == cudaSuccess && pa.devicePointer &&
                         (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged ||
                          pa.type == cudaMemoryTypeHost);
        cudaGetLastError();
        if (dev) {
            r->edges = static_cast<const int32_t *>(pa.devicePointer);
        } else {  // pageable memory: copy into the slot's pinned staging
            if (sv->stage_cap[slot] < B) {
                if (sv->stage[slot]) cudaFreeHost(sv->stage[slot]);
                sv->stage[slot] = nullptr;
                sv->stage_cap[slot] = 0;
                const int64_t cap = std::min<int64_t>(sv->max_batch, std::max<int64_t>(2 * B, 1 << 16));
                if (cudaHostAlloc((void **)&sv->stage[slot], sizeof(int32_t) * 2 * (size_t)cap, cudaHostAllocMapped) !=
                        cudaSuccess ||
                    cudaHostGetDevicePointer((void **)&sv->stage_dev[slot], sv->stage[slot], 0) != cudaSuccess) {
                    cudaGetLastError();
                    if (sv->stage[slot]) cudaFreeHost(sv->stage[slot]);
                    sv->stage[slot] = nullptr;
                    return set_status(PLDS_ENOMEM);
                }
                sv->stage_cap[slot] = cap;
            }
            std::memcpy(sv->stage[slot], edges, sizeof(int32_t) * 2 * (size_t)B);
            r->edges = sv->stage_dev[slot];
        }
    }
    if (op == kReqCoreness) {
        r->out = out_dev ? static_cast<double *>(out_devptr) : sv->qbuf_dev;
        sv->qdest[slot] = out_dev ? nullptr : out;
    }
    sv->need[slot] = need;
    sv->inflight_need += need;
    std::atomic_thread_fence(std::memory_order_release);
    *(volatile int32_t *)&r->state = kSlotReady;
    if (ticket) *ticket = sv->next_seq;
    sv->next_seq++;
    int rc = server_service(sv);
    if (rc) return set_status(rc);
    if (!sv->running) {
        rc = server_launch(sv);
        if (rc) return set_status(rc);
    }
    return set_status(PLDS_OK);
}

extern "C" int plds_server_configure(plds_server_t *sv, int64_t merge_max_edges, int64_t pool_limit_bytes) {
    if (!sv || pool_limit_bytes < 0 || merge_max_edges < -1) return set_status(PLDS_EINVAL);
    sv->merge_cap = merge_max_edges < 0 ? sv->max_batch : std::min(merge_max_edges, sv->max_batch);
    sv->pool_limit = pool_limit_bytes;
    return set_status(PLDS_OK);
}

extern "C" int32_t plds_opt_levels_per_group(int64_t m, double delta) {
    const int32_t r = opt_levels_per_group(m, delta);
    return r > 0 ? r : PLDS_EINVAL;
}

extern "C" int plds_server_admission(int64_t pool_cap, int64_t pool_used, int64_t inflight, int64_t need,
                                     int64_t free_bytes) {
    if (pool_cap < 0 || pool_used < 0 || inflight < 0 || need < 0 || free_bytes < 0) return PLDS_EINVAL;
    if (pool_cap - pool_used - inflight >= need) return 0;  // the pool has room
    // otherwise the pool must grow: a compacting grow needs a new pool that holds
    // every slot in use or promised, and it must fit in the free bytes
    if ((pool_used + inflight + need) <= free_bytes / 4) return 0;
    return inflight > 0 ? 1 : 2;
}

extern "C" int plds_server_poll(plds_server_t *sv, plds_request_result *out, int32_t cap) {
    if (!sv || (cap > 0 && !out) || cap < 0) return set_status(PLDS_EINVAL);
    server_collect(sv);
    int rc = server_service(sv);
    if (rc) return set_status(rc);
    const int32_t k = std::min<int32_t>(cap, (int32_t)sv->finished.size());
    for (int32_t i = 0; i < k; ++i) out[i] = sv->finished[i];
    sv->finished.erase(sv->finished.begin(), sv->finished.begin() + k);
    set_status(PLDS_OK);
    return k;
}

extern "C" int plds_server_drain(plds_server_t *sv) {
    if (!sv) return set_status(PLDS_EINVAL);
    const auto t0 = std::chrono::steady_clock::now();
    while (sv->done_seq < sv->next_seq) {
        server_collect(sv);
        int rc = server_service(sv);
        if (rc) return set_status(rc);
        if (std::chrono::steady_clock::now() - t0 > std::chrono::nanoseconds(sv->h->wait_limit_ns))
            return set_status(PLDS_ETIMEOUT);
    }
    return set_status(PLDS_OK);
}

extern "C" void plds_server_destroy(plds_server_t *sv) {
    if (!sv) return;
    plds_server_drain(sv);
    // wait for the loop to go idle and exit
    if (sv->running) cudaEventSynchronize(sv->done);
    sv->running = false;
    ServeCtl c{};
    if (cudaMemcpy(&c, sv->sc.p, sizeof(ServeCtl), cudaMemcpyDeviceToHost) == cudaSuccess)
        sv->h->stamp_base = c.stamp_next;
    cudaGetLastError();
    server_free(sv);
}
