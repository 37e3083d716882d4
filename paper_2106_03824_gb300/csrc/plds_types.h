// Internal structures shared by the host runtime and the device code of the GB300
// PLDS library (not part of the public C ABI).
#pragma once
#include <cstdint>

namespace pl {

constexpr int32_t kEmpty = -1;          // hash slot never used since the last rebuild
constexpr int32_t kTomb = -2;           // hash slot of a deleted neighbour
// Insertion rounds mark the movers of level l in the level word with the flag of
// l's parity; the level itself is the word & kLevelMask.  Flags never survive a batch.
constexpr int32_t kFlagEven = 1 << 30;
constexpr int32_t kFlagOdd = 1 << 29;
constexpr int32_t kLevelMask = kFlagOdd - 1;
constexpr int32_t kInf = 0x7fffffff;
constexpr int kMaxGroups = 512;        // groups (t+1) supported by the device tables
constexpr int kWindow = 256;           // desire-level histogram window (levels)
constexpr int kWarpHist = 512;         // per-warp shared histogram ints (>= kMaxGroups, kWindow)

// device error bits
enum : int32_t {
    kErrInvalidId = 1,
    kErrNeedPool = 2,
    kErrTimeout = 4,
    kErrInternal = 8,
    kErrListOverflow = 16,
};

// statistics slots (Ctl::st)
enum : int {
    kStSubmitted = 0, kStSelfLoops, kStDuplicates, kStFiltered, kStValid, kStRounds, kStMoves,
    kStVisits, kStDlEvals, kStDlVisits, kStSlotsScanned, kStUpVisits, kStAffected,
    kStSkipRounds, kStSkipMoves, kStSkipVisits, kStSkipUpVisits, kStCount
};

enum : int32_t { kOpInsert = 0, kOpDelete = 1 };

// Control words of one graph, in device memory.
struct Ctl {
    unsigned long long bar_arrivals;  // grid barrier: arrivals since launch (never reset within one)
    int32_t err;          // kErr* bits
    unsigned long long ucount;   // unique canonical keys
    unsigned long long vcount;   // valid (applied) keys
    int32_t tcount;              // touched vertices
    unsigned long long grow_total;  // slots requested by growing tables
    unsigned long long ltop[3];  // insertion: int4 units handed out of each up-list buffer
    int32_t imcnt[3];     // insertion: movers marked for a phase (phase index mod 3)
    int32_t itl[3];       // insertion: thread-mode scan items of a phase
    int32_t icl[3];       // insertion: chunk scan items of a phase
    // insertion, per phase (index mod 3), about the movers of level l that climb on
    // to l + 1: how many; kInf minus their smallest new up-degree; their degree and
    // new up-degree sums; kInf minus the lowest level >= l + 1 of a neighbour of a
    // mover of l that is not itself a mover (complements, so that zero means none)
    int32_t icont[3];
    int32_t iminup_c[3];
    int32_t ilow_c[3];
    unsigned long long isdeg[3];
    unsigned long long isup[3];
    // insertion, jump variant: pending violators in P[i] (the list in use) and,
    // per round parity, kInf minus their lowest level (0: none); movers of a round
    // (index mod 3, in TL) and those with large tables (round parity, in M[0])
    int32_t jpend[2];
    int32_t jcons[2];     // jump variant: entries of P[i] already taken (marked in place)
    int32_t jnext_c[2];
    int32_t jmov[3];
    int32_t jbig[2];
    // jump variant, per round parity, for skipping pure rounds: movers still
    // violating at their target; movers whose target is not l + 1; kInf minus the
    // lowest level of a pending entry that is not such a mover, of a neighbour of a
    // mover that is no mover (>= l + 1), and of the staying movers' up-degree; the
    // staying movers' degree sum
    int32_t jstay[2];
    int32_t jnonunit[2];
    int32_t jother_c[2];
    int32_t jlow_c[2];
    int32_t jminup_c[2];
    unsigned long long jsdeg[2];
    int32_t mcnt[2];      // table growth / deletion movers
    int32_t tlcnt[2];     // thread-mode movers
    int32_t clcnt[2];     // chunk items
    int32_t nlev;         // number of distinct initial-candidate levels
    int32_t pcnt[2];      // deletion pending list sizes
    int32_t rcnt[2];      // deletion recompute list sizes
    int32_t nextmin[2];   // deletion: smallest pending desire-level
    int32_t err_site;     // which check raised the first error (0 = none)
    int32_t err_info[3];  // values seen by that check (diagnostics)
    int32_t trace_n;      // per-round records written
    int32_t rbcnt;        // violators with large tables (block-wide desire-level)
    // steps before the rounds: list lengths and room reserved once per block
    unsigned long long ttotal;  // touched vertices
    unsigned long long gtotal;  // growing tables (insert) / warp shrink list (delete)
    unsigned long long btotal;  // block shrink list
    unsigned long long atotal;  // shrink arena ints
    unsigned long long ctotal;  // chunks of the old tables of growing vertices / of large tables to shrink
    unsigned long long c1total;  // chunks of the large shrinking tables' new slots (clear)
    unsigned long long c2total;  // chunks of their live keys (reinsert)
    unsigned long long pool_old;  // pool top before the growing tables took their room
    // diagnostics (trace mode): per phase parity, the latest and earliest time a block
    // finished its share of an insertion phase
    unsigned long long tw_max[2];
    unsigned long long tw_min_c[2];  // complement of the earliest time (zero means none)
    unsigned long long st[kStCount];
};

// Everything a device routine needs to know about one graph and its current batch.
struct GraphCtx {
    int32_t n, Lg, K, G;
    int32_t op;            // kOpInsert / kOpDelete
    int32_t stamp_base;    // stamps of this batch are stamp_base + 1 .. stamp_base + K + 1
    int32_t thread_max_cap;
    int32_t load_num, load_den;
    int32_t test_delay_us;
    int32_t barrier_sleep_ns;
    int32_t block_cap;     // tables above this many slots get a whole block (desire-levels, rebuilds)
    int32_t list_cap;      // insertion: chunk-scanned tables from this size on get an up-list
    int32_t jump;          // insertion violators move straight to their targets (jump variant)
    int32_t pre_done;      // the steps before the rounds ran as separate kernels (plain form)
    int32_t pad3;
    int64_t wait_limit_ns;
    const int32_t *upmax;  // [G]
    const int32_t *dnmin;  // [G]
    int32_t *level, *deg, *up, *upstar;   // [n]
    int64_t *off;          // [n] first slot of the vertex's table in the pool
    int32_t *cap;          // [n] table size (power of two >= 4, or 0)
    int32_t *tomb;         // [n] tombstones in the table
    int32_t *stamp;        // [n] dedupe stamps
    int32_t *dlv;          // [n] pending desire-level, -1 when none
    int32_t *dslack;       // [n] deletion: slack of a pending vertex's desire-level (see dl_batch)
    int32_t *inc;          // [n] incoming insertions of the batch
    int32_t *slots;        // adjacency pool
    unsigned long long *pool_top;  // slots handed out
    int64_t pool_cap;
    // batch input and scratch
    const int32_t *edges;  // int32[B][2]
    int64_t B;
    unsigned long long *hset;  // batch key set, hcap entries (power of two), all ones = empty
    int64_t hcap;
    unsigned long long *ukeys;  // unique keys [B]
    unsigned long long *vkeys;  // valid keys [B]
    int32_t *touched;      // touched vertices [tcap]
    int32_t *S;            // candidates sorted by level [tcap]
    int32_t *bins;         // [K+1] level histogram / offsets
    int32_t *levlist;      // [K] distinct candidate levels
    unsigned long long *acc;  // [n] insertion: per mover {chunks done << 32 | neighbours left below}
    int32_t *lbuf[3];      // insertion: up-list buffers (phase index mod 3), lcap entries each
    int64_t lcap;
    int32_t *lout;         // [n] insertion: a chunk-mode mover's output up-list (int4 units), -1 none
    int32_t *lfill[2];     // [n] insertion: entries written to it so far (by phase parity)
    int4 *M[2];            // movers {v, aux, cap, -} [n]
    int4 *TL[3];           // thread-mode scan items {v, log2 cap, offset/4, aux} [n]
    int4 *CL[3];           // chunk scan items {v, chunk<<5 | log2 cap, offset/4, aux} [clcap]
    int64_t clcap;
    int4 *P[2];            // pending {v, dl, -, -} [2n]
    int32_t *R[2];         // desire-level recompute candidates; R[1]: violators to evaluate [n]
    int32_t *arena;        // table-shrink scratch
    int64_t arena_cap;
    int32_t *trace;        // per-round diagnostics records (8 int32 each) or null
    int32_t trace_cap;
    Ctl *ctl;
};

// The per-batch inputs of one batch: kept apart from the graph's context so that a
// loop applying many batches to one graph can keep that context in kernel
// parameter space.
struct BatchIn {
    const int32_t *edges;  // int32[B][2]
    int64_t B;
    int32_t op;            // kOpInsert / kOpDelete
    int32_t stamp_base;    // stamps of this batch are stamp_base + 1 .. stamp_base + K + 1
};

}  // namespace pl
