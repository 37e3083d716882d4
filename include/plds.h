/*
 * plds.h -- C ABI of the GB300 (sm_103a) parallel level data structure (PLDS).
 *
 * The library maintains, for an undirected graph on vertex ids [0, n), the levels
 * of the PLDS of Liu, Shi, Yu, Dhulipala and Shun (SPAA'22, "Parallel
 * Batch-Dynamic Algorithms for k-Core Decomposition and Related Graph Problems"),
 * and from them (2+3/lambda)(1+delta)-approximate coreness estimates, under batches
 * of edge insertions and deletions.  All state lives in GPU memory; every step of a
 * batch (preprocessing, adjacency update, counters, level rounds) runs in the
 * library's own CUDA kernels.
 *
 * Conventions for every call:
 *   - Return value: PLDS_OK (0) or a negative PLDS_E* code.  plds_last_status()
 *     returns the code of the calling thread's last call.
 *   - Pointers to caller buffers (edges, out) may be host or device pointers; the
 *     library detects which.  Device pointers must be valid on the handle's device
 *     and are used in order on the handle's stream; host pointers are copied
 *     before the call returns.  The caller keeps ownership of its buffers.
 *   - Edge arrays are int32[B][2] (u, v pairs, row-major, 8 bytes per edge).
 *   - A handle is used by one host thread and one stream at a time.
 *   - After PLDS_ETIMEOUT or PLDS_EDEVICE the handle is poisoned: every further
 *     call except plds_destroy returns PLDS_EPOISONED.
 */
#ifndef PLDS_H
#define PLDS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PLDS_OK 0
#define PLDS_EINVAL (-1)     /* bad argument: n, delta, lambda, an id outside [0,n), NULL */
#define PLDS_ENOMEM (-2)     /* device memory could not be obtained; state unchanged */
#define PLDS_ETIMEOUT (-3)   /* a bounded device-side wait expired; handle poisoned */
#define PLDS_EDEVICE (-4)    /* CUDA reported an error; handle poisoned */
#define PLDS_EINTERNAL (-5)  /* an internal consistency check failed */
#define PLDS_EPOISONED (-6)  /* handle unusable after an earlier ETIMEOUT/EDEVICE */

typedef struct plds plds_t;

/* Device allocator used for every allocation of a handle.  alloc returns a device
 * pointer (NULL on failure) usable on `stream`; free releases it.  Either function
 * may be called from any library call on the handle's host thread. */
typedef struct plds_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} plds_allocator;

/* Statistics of the handle's last batch call (counts of the method's own work). */
typedef struct plds_stats {
    int64_t submitted;   /* edges passed in */
    int64_t self_loops;  /* dropped: u == v */
    int64_t duplicates;  /* dropped: repeated (min,max) key in the batch */
    int64_t filtered;    /* dropped: insert of a present / delete of an absent edge */
    int64_t valid;       /* updates applied */
    int64_t rounds;      /* levels at which at least one vertex moved */
    int64_t moves;       /* level changes (insert: one level each; delete: one per vertex) */
    int64_t visits;      /* neighbours of moving vertices: the sum of their degrees over the moves */
    int64_t dl_evals;    /* desire-level computations */
    int64_t dl_visits;   /* neighbours scanned by desire-level computations */
    int64_t slots_scanned; /* entries read by the level rounds (table slots: live, empty,
                              tombstone; up-list entries) */
    int64_t pool_slots_used;
    int64_t pool_slots_cap;
    int64_t device_bytes;  /* device memory currently held by the handle */
    int64_t pool_grows;    /* adjacency pool reallocations so far */
    int64_t err_bits;      /* device error word of the last call (diagnostics) */
    int64_t err_site;      /* internal check that raised it (diagnostics) */
    int64_t err_info[3];   /* values seen by that check (diagnostics) */
    int64_t kernel_ns;     /* device time of the last call's launch sequence: step kernels and
                              level-rounds kernel, summed over its attempts (CUDA events) */
    int64_t launches;      /* kernels launched by this handle since creation */
    int64_t up_visits;     /* insertion: up-neighbours of moving vertices, the sum of their
                              up-degrees over the moves (what a move must examine) */
    int64_t affected;      /* neighbours whose up- or up*-degree a move changed, summed over
                              the moves (the counter updates the moves made) */
    /* Insertion rounds that change nothing but the level of the same climbing set
       (no neighbour outside the set on the levels passed, no other candidate) are
       counted, not run: of the rounds, moves, visits and up_visits above, these
       many belong to such skipped rounds. */
    int64_t skipped_rounds;
    int64_t skipped_moves;
    int64_t skipped_visits;
    int64_t skipped_up_visits;
    int64_t pre_ns;        /* device time of the last call's steps before the level rounds
                              (preprocessing, table growth/shrinking, adjacency and counter
                              updates; part of kernel_ns) */
} plds_stats_t;

/* Tuning knobs: they change speed only, never results. Zero fields keep defaults. */
typedef struct plds_tuning {
    int32_t thread_max_cap;   /* tables up to this many slots are scanned by one thread (0 = default:
                                 8 for deletion batches and insertion batches of at most 300,000
                                 edges, 16 for larger insertion batches and the serving loop) */
    int32_t load_num;         /* a table grows when live+tombstones+incoming > cap*load_num/load_den */
    int32_t load_den;
    int32_t block_threads;    /* threads per block of the batch kernel (multiple of 32, 128..512) */
    int32_t blocks_per_sm;    /* resident blocks per SM for the cooperative kernel */
    int32_t test_delay_us;    /* testing only: block 0 sleeps this long before its first barrier
                                 (exercises the bounded waits); 0 in normal use */
    int32_t trace_rounds;     /* diagnostics: 1 = record one line per level round (plds_trace) */
    int32_t barrier_sleep_ns; /* pause between polls of a grid-barrier wait (0 = default 32, -1 = none) */
    int32_t block_cap;        /* tables above this many slots get a whole block for desire-levels
                                 and rebuilds, smaller ones a warp (0 = default: 1024 for a
                                 handle, 4096 for the graphs of a set; else >= 4) */
    int32_t track_orientation; /* 1 = every plds_batch_insert / plds_batch_delete call saves the
                                  levels at its start (4n bytes of device memory and one copy)
                                  so that plds_flips / plds_oriented_updates can report it */
    int32_t list_cap;         /* insertion: a moving vertex whose table has at least this many
                                 slots keeps the neighbours still on its level or above in an
                                 up-list for its next move (0 = default 256; 2^30 = never) */
} plds_tuning;

/*
 * Create an empty PLDS on the current CUDA device: n vertices on level 0, no edges.
 * delta > 0 and lambda > 0 are the paper's constants (defaults 0.4 and 3); they are
 * converted to rationals with denominator 10^6.  Levels per group follow the
 * paper's Section "Detailed PLDS Algorithm": 4*ceil(log_{1+delta} n) (taken as
 * 4*max(1,t) with t the smallest integer such that (1+delta)^t >= n), groups 0..t.
 * Returns NULL on error (plds_last_status() says which).
 */
plds_t *plds_create(int32_t n, double delta, double lambda);

/*
 * As plds_create, plus: levels_per_group (0 = the paper's 4*ceil(log_{1+delta} n);
 * a positive value overrides it), allocator (NULL = cudaMallocAsync/cudaFreeAsync),
 * stream (a cudaStream_t; NULL = the legacy default stream), flags (0, or a sum of:
 * PLDS_FLAG_HEURISTIC: Invariant 1's coefficient 2 + 3/lambda replaced by 1.1, the
 * experiments section's "heuristic parameters" -- both invariants still hold, the
 * efficiency and approximation bounds do not;
 * PLDS_FLAG_JUMP: insertion batches take the Experiments section's implementation
 * variant ("filter and sort" desire-levels for the vertices moved up, read as: each
 * round, every violator of Invariant 1 on the lowest level l that holds one moves at
 * once to the lowest level above l on which it satisfies Invariant 1 with every
 * other vertex where it is) instead of Algorithm 2's one level per round -- the
 * levels after every batch are Algorithm 2's, the rounds and moves statistics are
 * the variant's; deletions are unchanged;
 * other bits: PLDS_EINVAL).
 */
#define PLDS_FLAG_HEURISTIC 1u
#define PLDS_FLAG_JUMP 2u
plds_t *plds_create_ex(int32_t n, double delta, double lambda, int32_t levels_per_group,
                       const plds_allocator *allocator, void *stream, uint32_t flags);

/*
 * Apply a batch of edge insertions: Algorithm 1's insertion half, i.e. batch
 * preprocessing (framework section: drop self-loops, keep one copy per (min,max)
 * key, drop insertions of edges already present) followed by RebalanceInsertions
 * (Algorithm 2): levels processed bottom-up, every vertex violating Invariant 1
 * moves up one level per round.  Ids outside [0,n) reject the whole call with
 * PLDS_EINVAL before anything changes.  B == 0 is a no-op.  Blocks until done.
 */
int plds_batch_insert(plds_t *h, const int32_t *edges, int64_t B);

/*
 * Apply a batch of edge deletions: preprocessing (drop deletions of absent
 * edges) followed by RebalanceDeletions (Algorithm 3) with desire-levels
 * (Definition "Desire-level", computed as Algorithm 4 does: the level closest
 * below at which Invariant 2 holds).  Each vertex moves at most once, down.
 * Same error behaviour as plds_batch_insert.
 */
int plds_batch_delete(plds_t *h, const int32_t *edges, int64_t B);

/*
 * Allocation-free variant of plds_batch_insert (is_delete = 0) and
 * plds_batch_delete (is_delete = 1); the paper has no counterpart: it exists for
 * callers that must not allocate device memory while updating, such as a
 * latency-critical update loop (cudaMalloc can synchronise the whole device) or
 * a process with a fixed device-memory budget whose allocator cannot be called
 * from here.  Same batch semantics and results as the regular calls.
 *   - Uses only the handle's arrays plus one library-wide device array of 4 MiB
 *     (held by every GPU that loads the library until the process exits) for the
 *     per-batch scratch; no cudaMalloc, cudaFree or allocator callback is called.
 *   - B may be at most 65536 edges; larger batches return PLDS_EINVAL (use the
 *     regular calls).  If the adjacency pool has no room for the tables this
 *     batch needs, returns PLDS_ENOMEM with the graph unchanged (growing the pool
 *     would allocate; a regular call grows it).
 *   - The first call on a device looks up that array's device address; make that
 *     first call before any stream capture.
 *   - All calls, from every handle on a device, share the one array and it keeps
 *     the previous call's contents; calls that overlap on the GPU (another handle
 *     on another stream, another host thread) race and must be serialised by the
 *     caller.
 *   - These calls do not track orientation: after one, plds_flips and
 *     plds_oriented_updates return PLDS_EINVAL until the next regular batch call
 *     made with tuning.track_orientation set.
 *   - The looked-up address belongs to the device's current context: the library
 *     must not be used across a cudaDeviceReset of that device (the reset also
 *     invalidates every handle on it).
 */
int plds_batch_static(plds_t *h, const int32_t *edges, int64_t B, int32_t is_delete);

/*
 * Coreness estimate of every vertex (Definition "Coreness Estimate"):
 * (1+delta)^{max(floor((level+1)/L)-1, 0)} with L the levels per group, and 0 for a
 * vertex of degree 0.  out: double[n], host or device.
 */
int plds_coreness(plds_t *h, double *out);

/* The exponent of the estimate above per vertex (-1 for degree 0).  out: int32[n]. */
int plds_coreness_exponent(plds_t *h, int32_t *out);

/* Current level of every vertex.  out: int32[n], host or device. */
int plds_levels(plds_t *h, int32_t *out);

/* deg, up-degree and up*-degree counters (Section "Detailed PLDS Algorithm":
 * up = neighbours on levels >= level(v), up* = neighbours on levels >= level(v)-1).
 * Any pointer may be NULL.  Each: int32[n], host or device. */
int plds_counters(plds_t *h, int32_t *deg, int32_t *up, int32_t *upstar);

/* Statistics of the last batch call. */
int plds_stats(plds_t *h, plds_stats_t *out);

/* out[4] = {t, levels per group, groups, levels K}. */
int plds_params(plds_t *h, int32_t *out);

/* Per-group integer thresholds: upmax[i] = floor((2+3/lambda)(1+delta)^i) and
 * dnmin[i] = ceil((1+delta)^i), both clamped to n (Invariants 1 and 2).
 * Each array has `groups` entries (out[2] of plds_params).  Host pointers. */
int plds_tables(plds_t *h, int32_t *upmax, int32_t *dnmin);

/* Levels per group of the paper's optimised variant PLDSOpt (experiments
 * section, "Evaluated Algorithms"): ceil(log_{1+delta}(m) / 50), at least 1, for a
 * graph of about m edges -- pass it as levels_per_group to plds_create_ex.  Exact:
 * the smallest L >= 1 with (1+delta)^(50 L) >= m, delta read as a rational with
 * denominator 10^6.  m must be in [0, 2^32); returns PLDS_EINVAL otherwise or for
 * a delta so small that the test needs more than 20000 bits.  With fewer levels
 * per group the batch rules and both invariants are unchanged, but the
 * (2+3/lambda)(1+delta) approximation bound is no longer guaranteed. */
int32_t plds_opt_levels_per_group(int64_t m, double delta);

/*
 * Low out-degree orientation (Section "O(alpha) Out-Degree Orientation",
 * Algorithm 5).  An edge goes from the endpoint on the lower level to the one on
 * the higher level; on equal levels from the lower id to the higher id (the
 * reading of Algorithm 5's flip conditions; the section's prose states the
 * opposite tie rule).  Every vertex's out-degree is at most its up-degree, hence at
 * most the Invariant-1 cutoff of its level's group.  Edge arrays are int32[B][2],
 * outputs int32 arrays; host or device pointers.
 *   plds_orient: tail[i] = the endpoint edge i goes from, -1 if the edge is not in
 *     the graph or an id is out of range.
 *   plds_out_degrees: out[v] = number of edges going from v (int32[n]).
 *   plds_flips: F of the last batch call (which must have been a plds_batch_insert /
 *     plds_batch_delete made with tuning.track_orientation = 1, and the last call
 *     changing the graph): every edge present before and after it whose orientation
 *     changed, as (tail, head) BEFORE the flip.  Up to cap pairs go to out, in no
 *     particular order; *count gets the total.  PLDS_EINVAL if tracking was off.
 *   plds_oriented_updates: J of that call: its valid updates as (tail, head),
 *     insertions oriented after the call, deletions before it.
 */
int plds_orient(plds_t *h, const int32_t *edges, int64_t B, int32_t *tail);
int plds_out_degrees(plds_t *h, int32_t *out);
int plds_flips(plds_t *h, int32_t *out, int64_t cap, int64_t *count);
int plds_oriented_updates(plds_t *h, int32_t *out, int64_t cap, int64_t *count);

/*
 * Static (2+eps')-approximate k-core (Section "Static (2+eps)-Approximate k-Core",
 * Algorithm 6) of the handle's current graph; the levels are not touched.
 * Bucketed peeling with eps = (sqrt(4 eps' + 9) - 3) / 2 and delta = 2 / eps:
 * C[v] starts at deg(v), bucket(C) = ceil(log_{1+eps} C) (decided against the
 * table (1+eps)^b built by repeated multiplication in double); the outer loop takes
 * the lowest non-empty bucket as threshold index t; up to ceil(log_{1+delta} n)
 * inner iterations each peel the whole lowest bucket and set every surviving
 * neighbour's C = max(C - r, ceil((1+eps)^(t-1))) (r = its peeled neighbours) and
 * bucket = max(bucket(C), t), continuing while (1+eps)^next <= (2+eps)(1+eps)^t.
 * out[v] = (1+eps)^(v's bucket when peeled), 0 for isolated vertices (the worked
 * example's values); double[n], host or device.  stats (int64[3] or NULL): outer
 * iterations, inner iterations, neighbour visits.  PLDS_EINVAL for eps' <= 0.
 */
int plds_static_coreness(plds_t *h, double eps_prime, double *out, int64_t *stats);

/* Use another stream for subsequent calls. */
int plds_set_stream(plds_t *h, void *stream);

/* Replace tuning knobs (see plds_tuning); results are unaffected. */
int plds_set_tuning(plds_t *h, const plds_tuning *t);

/* Limit, in nanoseconds, of every device-side wait (grid barrier); 0 = default 20 s.
 * When a wait runs out the kernel stops, the call returns PLDS_ETIMEOUT. */
int plds_set_wait_limit(plds_t *h, int64_t ns);

/* Diagnostics: per-round records of the last batch call when tuning.trace_rounds
 * is set (single-graph calls).  Each record is 12 int32; times in nanoseconds from
 * the device clock.  Record 0: {-1 (insert) or -2 (delete), then the durations of
 * the steps between the rounds kernel's start and its first round; for a deletion
 * batch, entries 8-10 hold the touched vertices and how many of them took a
 * desire-level computation by a warp and by a block}.  Then one per
 * phase.  Insertion (Algorithm 2): {level, 1 = movers' scan or 0 = test of initial
 * candidates, movers, thread-mode items, chunk items, first block's work, its
 * publish + barrier, pure rounds skipped after the phase, latest and earliest end
 * of a block's work after the phase start, 0, 0}.  Deletion (Algorithm 3): {level,
 * pending entries, movers, thread-mode items, chunk items, take, apply and
 * desire-level parts seen by the first block, desire-levels computed by a warp and
 * by a block after the classifying pass, 0, 0}.  Jump variant: {level, 2,
 * movers, large-table movers, pending left, round time, its first part, pure
 * rounds skipped, staying movers, movers with a non-unit target, lowest other
 * pending level or -1, lowest non-mover neighbour level or -1}.
 * out holds cap records;
 * returns the number of records written, or a negative PLDS_E* code. */
int plds_trace(plds_t *h, int32_t *out, int32_t cap);

/*
 * Batched form: a set of independent graphs updated together, one kernel launch
 * per round (the paper has no counterpart; it batches many small graphs whose
 * rounds are too short to fill the GPU one at a time).  Each graph behaves
 * exactly as a handle of its own: a round applies to graph i its insertion half
 * and then its deletion half (Algorithm 1), and the resulting state equals that
 * of plds_batch_insert followed by plds_batch_delete on that graph alone.
 *   plds_set_create: count graphs with n[i] vertices each (delta, lambda,
 *     allocator, stream as in plds_create_ex).  NULL on error.
 *   plds_set_update: edges holds all halves back to back as int32 pairs, host or
 *     device; offsets has 2*count+1 entries (in edges, not ints): graph i's
 *     insertion half is pairs [offsets[2i], offsets[2i+1]) and its deletion half
 *     [offsets[2i+1], offsets[2i+2]).  Blocks until done.  Errors as the single
 *     calls; an id outside [0, n[i]) rejects the round before graph i changes.
 *   plds_set_graph: the handle of graph i, owned by the set, for queries and
 *     statistics (the last round's counts of both halves, summed).
 * The graphs of a set start with thread_max_cap = 64 (a block per graph scans
 * small tables better one thread each); plds_set_tune / plds_set_autotune change it.
 */
typedef struct plds_set plds_set_t;
plds_set_t *plds_set_create(int32_t count, const int32_t *n, double delta, double lambda,
                            const plds_allocator *allocator, void *stream);
int plds_set_update(plds_set_t *s, const int32_t *edges, const int64_t *offsets);
int plds_set_tune(plds_set_t *s, const plds_tuning *t);
int plds_set_autotune(plds_set_t *s, int32_t rounds, const int32_t *const *edges, const int64_t *const *offsets,
                      int32_t timed_from, int32_t max_trials, plds_tuning *best);
plds_t *plds_set_graph(plds_set_t *s, int32_t i);
void plds_set_destroy(plds_set_t *s);

/*
 * Autotuner (the paper has no counterpart: its cutoffs are a multicore design's).
 * The knobs that change only speed -- the thread cutoff (thread_max_cap), the
 * block cutoff (block_cap), the hash load factor (load_num/load_den) and the
 * up-list cutoff (list_cap) -- are picked by coordinate descent: starting from `start`, each knob in that order
 * takes every value of its candidate list with the others held, and keeps the
 * value of lowest cost (a new value must cost at least 2 % less than the
 * incumbent); passes repeat while one of them improves, within max_trials cost
 * evaluations.  Candidates: thread_max_cap {4, 8, 16, 32, 64}, block_cap {1024,
 * 2048, 4096, 8192, 16384}, load {1/2, 5/8, 3/4, 7/8}, list_cap {128, 256, 1024,
 * 2^30}.
 *   plds_tune_search: the search alone, against any cost function (no device use):
 *     cost(t, ctx) returns a cost (seconds) or a negative value to stop the search
 *     with PLDS_EINTERNAL.  *best gets the chosen knobs (the other fields of start
 *     are kept); returns the number of evaluations or a negative code.
 *   plds_set_tune: the same knobs for every graph of a set.
 *   plds_set_autotune: the search for a set, on a sample of its workload: each
 *     evaluation builds a scratch set of the same graph sizes, applies rounds
 *     0..rounds-1 (edges[r], offsets[r] as for plds_set_update; rounds before
 *     timed_from untimed, e.g. a preload) and costs the wall time of the rest.
 *     The set itself is not changed except that the best knobs are applied to it
 *     (and written to *best).
 */
typedef double (*plds_tune_cost)(const plds_tuning *t, void *ctx);
int plds_tune_search(const plds_tuning *start, plds_tune_cost cost, void *ctx, int32_t max_trials,
                     plds_tuning *best);

/*
 *   plds_autotune: the search for one handle, on a sample stream: each evaluation
 *     builds a scratch handle configured like h (n, delta, lambda, levels per
 *     group, flags, allocator, stream, the other tuning fields), applies batches
 *     0..nbatches-1 -- batch b is edges[offsets[b] .. offsets[b+1]) (int32 pairs,
 *     host or device; offsets has nbatches + 1 entries, in edges), an insertion if
 *     kinds[b] == 0, a deletion if 1 -- and costs the wall time of the batches from
 *     timed_from on (the earlier ones build the sample's state untimed).  h's graph
 *     is not touched; its knobs become the best ones (also written to *best when
 *     non-null).  PLDS_EINVAL on bad arguments; a failing sample batch's code
 *     otherwise.
 */
int plds_autotune(plds_t *h, const int32_t *edges, const int64_t *offsets, const int32_t *kinds, int32_t nbatches,
                  int32_t timed_from, int32_t max_trials, plds_tuning *best);

/*
 * Serving form: a device-resident request loop over one graph (the paper has no
 * counterpart).  One persistent kernel applies requests from a ring of `slots`
 * slots in pinned host memory, in submission order; coreness queries see the state
 * after every earlier request.  While a server is open on a handle, use only the
 * server calls on that handle.
 *
 * Continuous batching: requests that wait in the ring while the device works are
 * admitted together -- the loop applies a run of consecutive insertion requests
 * (or deletion requests) as ONE batch of at most `merge_max_edges` edges and 64
 * requests.  Every request of such a batch reports the batch's first ticket and
 * its number of requests (batch_first, batch_size), so the schedule can be
 * replayed batch by batch (for instance by a sequential implementation applying
 * the concatenated edges as one batch).  Merging changes which levels the
 * vertices end on, not the edge set, and every estimate keeps the (2+eps)
 * approximation bound (Section "Batch-Dynamic k-Core Decomposition", the
 * approximation lemma on the coreness estimate).  A request holding an id outside [0, n) is rejected alone
 * (status PLDS_EINVAL, nothing of it applied); the other requests of its batch are
 * applied.  With merge_max_edges = 0 every request is its own batch, and the
 * graph ends exactly as if each request had been its own plds_batch_insert /
 * plds_batch_delete call.
 *
 * Admission: a request is admitted when a ring slot is free and, for an insertion
 * of B edges, the adjacency can take its worst case (both endpoint tables of every
 * edge doubling: ceil(4 B den / num) slots at load num/den), either in the pool as
 * it is or in a grown pool that fits in free device memory (1 GiB kept free) and
 * in the pool limit.  Otherwise submit waits for admitted requests to finish, or
 * returns PLDS_ENOMEM (nothing admitted) when none is left to wait for.
 *
 *   plds_server_create: slots in the ring (1..4096); max_batch = largest batch
 *     (edges) of one request and of one merged batch.  Merging starts enabled
 *     with merge_max_edges = max_batch.
 *   plds_server_configure: merge_max_edges (0 = unchanged boundaries, -1 =
 *     max_batch; larger values are clamped to max_batch) and pool_limit_bytes
 *     (0 = no limit beyond free device memory).  Applies to requests submitted
 *     afterwards.
 *   plds_server_submit: op 0 insertion batch, 1 deletion batch, 2 coreness query
 *     (out = double[n], host or device; edges ignored).  Edge arrays may be device
 *     memory or pinned host memory (read in place by the running loop: their
 *     contents must be complete at submission -- no copy still in flight on a
 *     stream -- and unchanged until the request has finished) or pageable host
 *     memory (copied at submission).  Blocks only while every slot is busy or
 *     admission waits.  *ticket gets the request's number (0, 1, ...).
 *   plds_server_poll: copies up to cap finished requests into out (oldest first);
 *     returns their count or a negative code.
 *   plds_server_drain: waits until every submitted request has finished.
 *   plds_server_destroy: drains, stops the loop, frees the server (not the graph).
 *   plds_server_admission: the admission rule above as a pure function (no device
 *     use): pool_cap, pool_used, inflight (slots promised to admitted requests) and
 *     need in adjacency slots, free_bytes the device memory a grown pool may take.
 *     Returns 0 admit, 1 wait for admitted requests, 2 reject, or PLDS_EINVAL for a
 *     negative argument.
 */
typedef struct plds_server plds_server_t;
typedef struct plds_request_result {
    int64_t ticket;
    int32_t op;
    int32_t status;     /* PLDS_OK or a PLDS_E* code */
    int64_t valid;      /* updates applied by the request's batch */
    int64_t rounds;     /* of the request's batch */
    int64_t moves;      /* of the request's batch */
    int64_t device_ns;  /* time the device spent on the request's batch */
    int64_t batch_first;  /* ticket of the first request of the batch it was applied in */
    int32_t batch_size;   /* requests in that batch (1 when not merged) */
    int32_t pad;
    int64_t done_ns;      /* CLOCK_MONOTONIC time at which the host saw it finish */
} plds_request_result;
plds_server_t *plds_server_create(plds_t *h, int32_t slots, int64_t max_batch);
int plds_server_configure(plds_server_t *sv, int64_t merge_max_edges, int64_t pool_limit_bytes);
int plds_server_submit(plds_server_t *sv, int32_t op, const int32_t *edges, int64_t B, double *out,
                       int64_t *ticket);
int plds_server_poll(plds_server_t *sv, plds_request_result *out, int32_t cap);
int plds_server_drain(plds_server_t *sv);
void plds_server_destroy(plds_server_t *sv);
int plds_server_admission(int64_t pool_cap, int64_t pool_used, int64_t inflight, int64_t need,
                          int64_t free_bytes);

/* Status code of the calling thread's last call. */
int plds_last_status(void);

/* Free all device memory of the handle. */
void plds_destroy(plds_t *h);

#ifdef __cplusplus
}
#endif
#endif /* PLDS_H */
