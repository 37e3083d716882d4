/*
 * plds_oracle.c -- plain, slow, sequential CPU reference of the PLDS batch update
 * (Liu, Shi, Yu, Dhulipala, Shun: "Parallel Batch-Dynamic Algorithms for k-Core
 * Decomposition and Related Graph Problems", SPAA'22).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this
 * file; only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg load it.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it follows, section by section of the paper:
 *   - Levels, groups, Invariants 1 and 2, up / up* degrees, desire-level:
 *     Section "Detailed PLDS Algorithm" (Invariants 1-2, Definition of desire-level).
 *   - Update(B) = insertions then deletions: Algorithm 1.
 *   - RebalanceInsertions: Algorithm 2 (level-by-level, move violators up one level);
 *     with ORC_JUMP, the implementation variant of Section "Experiments" that moves
 *     each violator straight to a desire-level computed for it (see jump_target).
 *   - RebalanceDeletions: Algorithm 3, with the desire-level computed straight from
 *     its Definition (a downward linear scan testing both invariants), not with
 *     Algorithm 4's doubling search, so the device search is checked against a
 *     different method.
 *   - Batch preprocessing (keep unique updates; keep insertions of absent edges and
 *     deletions of present edges): Section "Batch-Dynamic Graph Problems" framework.
 *   - Coreness estimate: Definition "Coreness Estimate".
 *   - Exact coreness for checking the (2+3/lambda)(1+delta) bound: Matula-Beck
 *     bucket peeling (the textbook algorithm the paper cites for exact k-cores).
 *
 * Readings taken where the paper is silent or garbled (each is listed in the
 * repository's design notes):
 *   - levels per group L = 4*ceil(log_{1+delta} n), ceil taken exactly as the
 *     smallest t >= 0 with (1+delta)^t >= n, and L = 4*max(1,t);  groups 0..t.
 *   - thresholds become integers: up > c*x  <=>  up > floor(c*x);
 *     up* < x <=> up* < ceil(x); both clamped to n (degrees never exceed n-1).
 *   - delta and lambda are rationals with denominator 10^6.
 *   - all moves of one round happen first, then neighbour effects are evaluated on
 *     the post-move state (the paper's "same sequential order" lemma).
 *   - a vertex of degree 0 has coreness estimate 0.
 *
 * Counters up / up* are never stored: every use recomputes them from the
 * definition by scanning the neighbour list, which is slow but leaves nothing to
 * keep in sync.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_EINTERNAL -5

/* ------------------------------------------------------------------------- */
/* Exact rational arithmetic for the thresholds (little-endian base 2^32).   */
/* ------------------------------------------------------------------------- */
#define BN_LIMBS 400
typedef struct {
    uint32_t d[BN_LIMBS];
    int len; /* number of used limbs, 0 for zero */
} bignum;

static void bn_from(bignum *a, uint64_t v) {
    memset(a, 0, sizeof(*a));
    a->d[0] = (uint32_t)v;
    a->d[1] = (uint32_t)(v >> 32);
    a->len = a->d[1] ? 2 : (a->d[0] ? 1 : 0);
}

/* a *= m; returns 0, or -1 when the result no longer fits */
static int bn_mul_small(bignum *a, uint64_t m) {
    /* m < 2^32 is required by the callers */
    uint64_t carry = 0;
    for (int i = 0; i < a->len; ++i) {
        uint64_t cur = (uint64_t)a->d[i] * m + carry;
        a->d[i] = (uint32_t)cur;
        carry = cur >> 32;
    }
    int len = a->len;
    while (carry) {
        if (len >= BN_LIMBS) return -1;
        a->d[len++] = (uint32_t)carry;
        carry >>= 32;
    }
    a->len = len;
    while (a->len > 0 && a->d[a->len - 1] == 0) a->len--;
    return 0;
}

static int bn_cmp(const bignum *a, const bignum *b) {
    if (a->len != b->len) return a->len < b->len ? -1 : 1;
    for (int i = a->len - 1; i >= 0; --i)
        if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
    return 0;
}

/* compare k*Y with X */
static int bn_cmp_scaled(const bignum *Y, uint64_t k, const bignum *X, int *err) {
    static bignum t;
    t = *Y;
    if (bn_mul_small(&t, k)) { *err = 1; return 1; }
    return bn_cmp(&t, X);
}

/* floor(X / Y) clamped to `clamp` (X, Y > 0) */
static int64_t bn_floor_div_clamped(const bignum *X, const bignum *Y, int64_t clamp, int *err) {
    if (bn_cmp_scaled(Y, (uint64_t)clamp, X, err) <= 0) return clamp; /* clamp*Y <= X */
    int64_t lo = 0, hi = clamp;                                        /* lo*Y <= X < hi*Y */
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (bn_cmp_scaled(Y, (uint64_t)mid, X, err) <= 0) lo = mid; else hi = mid;
    }
    return lo;
}

/* ceil(X / Y) clamped to `clamp` (X, Y > 0) */
static int64_t bn_ceil_div_clamped(const bignum *X, const bignum *Y, int64_t clamp, int *err) {
    if (bn_cmp_scaled(Y, (uint64_t)clamp, X, err) < 0) return clamp; /* clamp*Y < X */
    int64_t lo = 0, hi = clamp;                                       /* lo*Y < X <= hi*Y */
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (bn_cmp_scaled(Y, (uint64_t)mid, X, err) < 0) lo = mid; else hi = mid;
    }
    return hi;
}

static int64_t gcd64(int64_t a, int64_t b) {
    while (b) { int64_t t = a % b; a = b; b = t; }
    return a;
}

/* delta or lambda given as a double becomes num/den with den = 10^6, reduced. */
static int to_rational(double x, int64_t *num, int64_t *den) {
    if (!(x > 0.0) || x > 1e6) return -1;
    double s = x * 1e6;
    int64_t nn = (int64_t)(s + 0.5);
    if (nn <= 0) return -1;
    int64_t dd = 1000000;
    int64_t g = gcd64(nn, dd);
    *num = nn / g;
    *den = dd / g;
    return 0;
}

/*
 * PLDSOpt's levels per group (experiments section, "Evaluated Algorithms", and the
 * implementation paragraph that divides the group size by 50): ceil(log_{1+delta}
 * m / 50), at least 1.  Decided exactly as the smallest L >= 1 with
 * (1+delta)^(50 L) >= m, i.e. (dnum+dden)^(50 L) >= m * dden^(50 L).
 * m must be below 2^32 and dnum+dden below 2^32; ORC_EINVAL otherwise, and when the
 * powers outgrow the bignum (very small delta).
 */
int32_t orc_opt_levels_per_group(int64_t m, double delta) {
    int64_t p, q;
    if (m < 0 || m > 0xffffffffLL || to_rational(delta, &p, &q) || p + q > 0xffffffffLL) return ORC_EINVAL;
    static bignum num, den, rhs;
    bn_from(&num, 1);
    bn_from(&den, 1);
    for (int32_t L = 1; L <= 1 << 20; ++L) {
        for (int k = 0; k < 50; ++k)
            if (bn_mul_small(&num, (uint64_t)(p + q)) || bn_mul_small(&den, (uint64_t)q)) return ORC_EINVAL;
        rhs = den;
        if (bn_mul_small(&rhs, (uint64_t)m)) return ORC_EINVAL;
        if (bn_cmp(&num, &rhs) >= 0) return L;
    }
    return ORC_EINVAL;
}

#define ORC_MAX_GROUPS 4096
#define ORC_MAX_LEVELS (1 << 24)

typedef struct {
    int32_t n;
    int64_t dnum, dden;   /* delta = dnum/dden */
    int64_t lnum, lden;   /* lambda = lnum/lden */
    int32_t t;            /* smallest t >= 0 with (1+delta)^t >= n */
    int32_t Lg;           /* levels per group */
    int32_t G;            /* groups 0..t */
    int32_t K;            /* levels 0..K-1 */
    int32_t *upmax;       /* [G]: floor((2+3/lambda)(1+delta)^i), clamped to n */
    int32_t *dnmin;       /* [G]: ceil((1+delta)^i), clamped to n */
} orc_tables;

/*
 * Group count and per-group thresholds (Invariants 1 and 2; group size from the
 * "Detailed PLDS Algorithm" section and the coreness-estimate Definition).
 */
/* flags: ORC_HEURISTIC replaces Invariant 1's coefficient 2 + 3/lambda by 1.1, the
   experiments' "heuristic parameters" (their efficiency bounds no longer hold). */
#define ORC_HEURISTIC 1
/* flags: ORC_JUMP takes the exact reading of the experiments' insertion variant
   ("a filter and sort that computes the desire-level of the vertices moved up"
   instead of moving them level by level): each round takes the lowest level l that
   holds a violator of Invariant 1, and every violator on l moves at once to its own
   target, the lowest level above l on which it would satisfy Invariant 1 with all
   other vertices where they are (jump_target).  Its levels equal Algorithm 2's:
   level assignments at or above the batch's starting levels under which every
   vertex satisfies Invariant 1 are closed under the pointwise minimum, so a least
   one exists; counts only grow as levels rise, so neither procedure moves a vertex
   past it, and both stop only when no vertex violates.  Rounds and moves differ. */
#define ORC_JUMP 2

static int build_tables(orc_tables *T, int32_t n, double delta, double lambda, int32_t lg_override,
                        int32_t flags) {
    memset(T, 0, sizeof(*T));
    if (n < 1) return ORC_EINVAL;
    if (to_rational(delta, &T->dnum, &T->dden)) return ORC_EINVAL;
    if (to_rational(lambda, &T->lnum, &T->lden)) return ORC_EINVAL;
    if (lg_override < 0 || (flags & ~(ORC_HEURISTIC | ORC_JUMP))) return ORC_EINVAL;
    T->n = n;
    int err = 0;
    /* t: smallest t with (dden+dnum)^t >= n * dden^t */
    static bignum P, Q, nQ;
    bn_from(&P, 1);
    bn_from(&Q, 1);
    int t = 0;
    for (;;) {
        nQ = Q;
        if (bn_mul_small(&nQ, (uint64_t)n)) return ORC_EINVAL;
        if (bn_cmp(&P, &nQ) >= 0) break;
        if (bn_mul_small(&P, (uint64_t)(T->dden + T->dnum))) return ORC_EINVAL;
        if (bn_mul_small(&Q, (uint64_t)T->dden)) return ORC_EINVAL;
        if (++t >= ORC_MAX_GROUPS) return ORC_EINVAL;
    }
    T->t = t;
    T->Lg = lg_override > 0 ? lg_override : 4 * (t > 1 ? t : 1);
    T->G = t + 1;
    int64_t K = (int64_t)T->G * T->Lg;
    if (K > ORC_MAX_LEVELS) return ORC_EINVAL;
    T->K = (int32_t)K;
    T->upmax = (int32_t *)malloc(sizeof(int32_t) * T->G);
    T->dnmin = (int32_t *)malloc(sizeof(int32_t) * T->G);
    if (!T->upmax || !T->dnmin) return ORC_ENOMEM;
    /* (2 + 3/lambda) = (2*lnum + 3*lden)/lnum, or 11/10 ; (1+delta)^i = (dden+dnum)^i / dden^i */
    uint64_t cnum = (uint64_t)(2 * T->lnum + 3 * T->lden), cden = (uint64_t)T->lnum;
    if (flags & ORC_HEURISTIC) {
        cnum = 11;
        cden = 10;
    }
    static bignum num, den, pw, qw;
    bn_from(&pw, 1);
    bn_from(&qw, 1);
    for (int i = 0; i < T->G; ++i) {
        num = pw;
        if (bn_mul_small(&num, cnum)) return ORC_EINVAL;
        den = qw;
        if (bn_mul_small(&den, cden)) return ORC_EINVAL;
        T->upmax[i] = (int32_t)bn_floor_div_clamped(&num, &den, n, &err);
        T->dnmin[i] = (int32_t)bn_ceil_div_clamped(&pw, &qw, n, &err);
        if (err) return ORC_EINVAL;
        if (i + 1 < T->G) {
            if (bn_mul_small(&pw, (uint64_t)(T->dden + T->dnum))) return ORC_EINVAL;
            if (bn_mul_small(&qw, (uint64_t)T->dden)) return ORC_EINVAL;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Graph storage: neighbour arrays + a map (u,v) -> slot in u's array.       */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint64_t *key; /* (u<<32)|v, EMPTY_KEY when free */
    int32_t *val;
    uint64_t cap;  /* power of two */
    uint64_t size;
} edge_map;

#define EMPTY_KEY 0xFFFFFFFFFFFFFFFFull

static uint64_t mix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

static int map_init(edge_map *m, uint64_t cap) {
    m->cap = cap;
    m->size = 0;
    m->key = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    m->val = (int32_t *)malloc(sizeof(int32_t) * cap);
    if (!m->key || !m->val) return -1;
    for (uint64_t i = 0; i < cap; ++i) m->key[i] = EMPTY_KEY;
    return 0;
}

static int64_t map_find(const edge_map *m, uint64_t k) {
    uint64_t i = mix64(k) & (m->cap - 1);
    for (;;) {
        if (m->key[i] == k) return (int64_t)i;
        if (m->key[i] == EMPTY_KEY) return -1;
        i = (i + 1) & (m->cap - 1);
    }
}

static int map_put(edge_map *m, uint64_t k, int32_t v);

static int map_grow(edge_map *m) {
    edge_map nm;
    if (map_init(&nm, m->cap * 2)) return -1;
    for (uint64_t i = 0; i < m->cap; ++i)
        if (m->key[i] != EMPTY_KEY) map_put(&nm, m->key[i], m->val[i]);
    free(m->key);
    free(m->val);
    *m = nm;
    return 0;
}

static int map_put(edge_map *m, uint64_t k, int32_t v) {
    if ((m->size + 1) * 2 > m->cap && map_grow(m)) return -1;
    uint64_t i = mix64(k) & (m->cap - 1);
    while (m->key[i] != EMPTY_KEY && m->key[i] != k) i = (i + 1) & (m->cap - 1);
    if (m->key[i] == EMPTY_KEY) m->size++;
    m->key[i] = k;
    m->val[i] = v;
    return 0;
}

/* remove by backward-shift deletion (linear probing, no tombstones) */
static void map_erase(edge_map *m, uint64_t k) {
    int64_t pos = map_find(m, k);
    if (pos < 0) return;
    uint64_t i = (uint64_t)pos, mask = m->cap - 1;
    m->key[i] = EMPTY_KEY;
    m->size--;
    uint64_t j = i;
    for (;;) {
        j = (j + 1) & mask;
        if (m->key[j] == EMPTY_KEY) return;
        uint64_t home = mix64(m->key[j]) & mask;
        /* move key[j] into the hole at i if its home is not in (i, j] cyclically */
        int in_range = (i <= j) ? (home > i && home <= j) : (home > i || home <= j);
        if (!in_range) {
            m->key[i] = m->key[j];
            m->val[i] = m->val[j];
            m->key[j] = EMPTY_KEY;
            i = j;
        }
    }
}

typedef struct {
    orc_tables T;
    int32_t n;
    int32_t *level;
    int32_t *deg;     /* number of neighbours = length of nbr[v] */
    int32_t *ncap;
    int32_t **nbr;
    edge_map map;
    /* scratch, all of size n */
    int32_t *stamp;   /* dedupe stamps */
    int32_t stamp_val;
    uint8_t *incident;
    uint8_t *marked;
    int32_t *dl;      /* desire-level while pending, else -1 */
    /* statistics of the last batch */
    int64_t st_submitted, st_selfloops, st_duplicates, st_filtered, st_valid;
    int64_t st_rounds, st_moves, st_visits, st_dl_evals, st_dl_visits;
    int32_t st_max_level_moves; /* insert: max levels one vertex climbed; delete: max moves of one vertex */
    int32_t st_dir_error;       /* 1 if a vertex moved against the batch's direction */
    int jump;                   /* ORC_JUMP: insertion violators move to their targets */
    /* orientation tracking (Algorithm 5): the last batch's levels before it, its
       kind and its valid (applied) edges */
    int track;
    int32_t *old_level;
    int last_op;                /* 0 insertion, 1 deletion, -1 none */
    uint64_t *last_keys;
    int64_t last_m;
} orc_plds;

static uint64_t ekey(int32_t u, int32_t v) { return ((uint64_t)(uint32_t)u << 32) | (uint32_t)v; }

static int nbr_push(orc_plds *h, int32_t u, int32_t v) {
    if (h->deg[u] == h->ncap[u]) {
        int32_t nc = h->ncap[u] ? 2 * h->ncap[u] : 4;
        int32_t *p = (int32_t *)realloc(h->nbr[u], sizeof(int32_t) * nc);
        if (!p) return -1;
        h->nbr[u] = p;
        h->ncap[u] = nc;
    }
    if (map_put(&h->map, ekey(u, v), h->deg[u])) return -1;
    h->nbr[u][h->deg[u]++] = v;
    return 0;
}

static void nbr_remove(orc_plds *h, int32_t u, int32_t v) {
    int64_t pos = map_find(&h->map, ekey(u, v));
    if (pos < 0) return;
    int32_t idx = h->map.val[pos];
    int32_t last = h->nbr[u][h->deg[u] - 1];
    h->nbr[u][idx] = last;
    if (last != v) h->map.val[map_find(&h->map, ekey(u, last))] = idx;
    h->deg[u]--;
    map_erase(&h->map, ekey(u, v));
}

static int has_edge(const orc_plds *h, int32_t u, int32_t v) {
    return map_find(&h->map, ekey(u, v)) >= 0;
}

/* group number of a level: levels [i*Lg, (i+1)*Lg - 1] form group i */
static int32_t gn(const orc_plds *h, int32_t l) { return l / h->T.Lg; }

/* up(v): neighbours in Z_{level(v)} (levels >= level(v)) -- by definition */
static int32_t up_of(const orc_plds *h, int32_t v) {
    int32_t c = 0, lv = h->level[v];
    for (int32_t i = 0; i < h->deg[v]; ++i) c += h->level[h->nbr[v][i]] >= lv;
    return c;
}

/* up*(v): neighbours in Z_{level(v)-1} -- by definition */
static int32_t upstar_of(const orc_plds *h, int32_t v) {
    int32_t c = 0, lv = h->level[v] - 1;
    for (int32_t i = 0; i < h->deg[v]; ++i) c += h->level[h->nbr[v][i]] >= lv;
    return c;
}

/* Invariant 1 for v at its current level: up(v) <= (2+3/lambda)(1+delta)^{gn(level)} */
static int inv1_ok(const orc_plds *h, int32_t v) {
    return up_of(h, v) <= h->T.upmax[gn(h, h->level[v])];
}

/* Invariant 2 for v at its current level: level > 0 => up*(v) >= (1+delta)^{gn(level-1)} */
static int inv2_ok(const orc_plds *h, int32_t v) {
    if (h->level[v] == 0) return 1;
    return upstar_of(h, v) >= h->T.dnmin[gn(h, h->level[v] - 1)];
}

/*
 * Desire-level (Definition): the level l' closest to level(v) at which v would
 * satisfy both invariants.  Only called for vertices that violate Invariant 2,
 * for which every admissible level lies below level(v); the scan goes from
 * level(v)-1 downwards and tests both invariants literally, with
 * cnt(x) = |N(v) ∩ Z_x| taken from a histogram of neighbour levels.
 */
static int32_t desire_level(orc_plds *h, int32_t v, int32_t *hist) {
    int32_t lv = h->level[v];
    h->st_dl_evals++;
    h->st_dl_visits += h->deg[v];
    for (int32_t x = 0; x <= lv + 1; ++x) hist[x] = 0;
    for (int32_t i = 0; i < h->deg[v]; ++i) {
        int32_t lw = h->level[h->nbr[v][i]];
        hist[lw < lv ? lw : lv]++;
    }
    /* suffix sums: hist[x] becomes cnt(x) = #neighbours with level >= x, for x <= lv */
    for (int32_t x = lv - 1; x >= 0; --x) hist[x] += hist[x + 1];
    for (int32_t lp = lv - 1; lp >= 0; --lp) {
        int inv2 = (lp == 0) || hist[lp - 1] >= h->T.dnmin[gn(h, lp - 1)];
        int inv1 = hist[lp] <= h->T.upmax[gn(h, lp)];
        if (inv1 && inv2) return lp;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Public API (ctypes)                                                        */
/* ------------------------------------------------------------------------- */
void orc_destroy(orc_plds *h);

int orc_tables_query(int32_t n, double delta, double lambda, int32_t lg_override, int32_t flags,
                     int32_t *out_t, int32_t *out_Lg, int32_t *out_G, int32_t *out_K,
                     int32_t *upmax, int32_t *dnmin, int32_t cap) {
    orc_tables T;
    int rc = build_tables(&T, n, delta, lambda, lg_override, flags);
    if (rc == ORC_OK) {
        *out_t = T.t;
        *out_Lg = T.Lg;
        *out_G = T.G;
        *out_K = T.K;
        for (int i = 0; i < T.G && i < cap; ++i) {
            upmax[i] = T.upmax[i];
            dnmin[i] = T.dnmin[i];
        }
    }
    free(T.upmax);
    free(T.dnmin);
    return rc;
}

orc_plds *orc_create_ex(int32_t n, double delta, double lambda, int32_t lg_override, int32_t flags) {
    orc_plds *h = (orc_plds *)calloc(1, sizeof(orc_plds));
    if (!h) return NULL;
    if (build_tables(&h->T, n, delta, lambda, lg_override, flags) != ORC_OK) {
        free(h->T.upmax);
        free(h->T.dnmin);
        free(h);
        return NULL;
    }
    h->n = n;
    h->level = (int32_t *)calloc(n, sizeof(int32_t)); /* every vertex starts on level 0 */
    h->deg = (int32_t *)calloc(n, sizeof(int32_t));
    h->ncap = (int32_t *)calloc(n, sizeof(int32_t));
    h->nbr = (int32_t **)calloc(n, sizeof(int32_t *));
    h->stamp = (int32_t *)calloc(n, sizeof(int32_t));
    h->incident = (uint8_t *)calloc(n, 1);
    h->marked = (uint8_t *)calloc(n, 1);
    h->dl = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!h->level || !h->deg || !h->ncap || !h->nbr || !h->stamp || !h->incident || !h->marked ||
        !h->dl || map_init(&h->map, 1024)) {
        orc_destroy(h);
        return NULL;
    }
    for (int32_t i = 0; i < n; ++i) h->dl[i] = -1;
    h->last_op = -1;
    h->jump = (flags & ORC_JUMP) != 0;
    return h;
}

orc_plds *orc_create(int32_t n, double delta, double lambda, int32_t lg_override) {
    return orc_create_ex(n, delta, lambda, lg_override, 0);
}

void orc_destroy(orc_plds *h) {
    if (!h) return;
    if (h->nbr)
        for (int32_t i = 0; i < h->n; ++i) free(h->nbr[i]);
    free(h->nbr);
    free(h->level);
    free(h->deg);
    free(h->ncap);
    free(h->stamp);
    free(h->incident);
    free(h->marked);
    free(h->dl);
    free(h->map.key);
    free(h->map.val);
    free(h->old_level);
    free(h->last_keys);
    free(h->T.upmax);
    free(h->T.dnmin);
    free(h);
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int32_t next_stamp(orc_plds *h) {
    if (h->stamp_val == INT32_MAX) {
        memset(h->stamp, 0, sizeof(int32_t) * h->n);
        h->stamp_val = 0;
    }
    return ++h->stamp_val;
}

/*
 * Batch preprocessing: reject ids outside [0,n) before any change; drop self-loops;
 * key each edge as (min,max); keep one copy of each key; keep insertions of absent
 * edges (want_present=0) or deletions of present edges (want_present=1).
 * Returns the number of kept keys in *out (malloc'ed), or a negative error.
 */
static int64_t preprocess(orc_plds *h, const int32_t *edges, int64_t B, int want_present, uint64_t **out) {
    h->st_submitted = B;
    h->st_selfloops = h->st_duplicates = h->st_filtered = h->st_valid = 0;
    for (int64_t i = 0; i < B; ++i) {
        int32_t u = edges[2 * i], v = edges[2 * i + 1];
        if (u < 0 || u >= h->n || v < 0 || v >= h->n) return ORC_EINVAL;
    }
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (B > 0 ? B : 1));
    if (!keys) return ORC_ENOMEM;
    int64_t nk = 0;
    for (int64_t i = 0; i < B; ++i) {
        int32_t u = edges[2 * i], v = edges[2 * i + 1];
        if (u == v) { h->st_selfloops++; continue; }
        keys[nk++] = u < v ? ekey(u, v) : ekey(v, u);
    }
    qsort(keys, (size_t)nk, sizeof(uint64_t), cmp_u64);
    int64_t m = 0;
    for (int64_t i = 0; i < nk; ++i) {
        if (i > 0 && keys[i] == keys[i - 1]) { h->st_duplicates++; continue; }
        int32_t u = (int32_t)(keys[i] >> 32), v = (int32_t)(keys[i] & 0xFFFFFFFFu);
        if (has_edge(h, u, v) != want_present) { h->st_filtered++; continue; }
        keys[m++] = keys[i];
    }
    h->st_valid = m;
    *out = keys;
    return m;
}

typedef struct { int32_t *a; int32_t len, cap; } ivec;
static int iv_push(ivec *v, int32_t x) {
    if (v->len == v->cap) {
        int32_t nc = v->cap ? 2 * v->cap : 16;
        int32_t *p = (int32_t *)realloc(v->a, sizeof(int32_t) * nc);
        if (!p) return -1;
        v->a = p;
        v->cap = nc;
    }
    v->a[v->len++] = x;
    return 0;
}

static void reset_stats(orc_plds *h) {
    h->st_rounds = h->st_moves = h->st_visits = h->st_dl_evals = h->st_dl_visits = 0;
    h->st_max_level_moves = 0;
    h->st_dir_error = 0;
}

/*
 * RebalanceInsertions (Algorithm 2).  Level l runs from 0 to K-1; at each level the
 * candidates are the vertices on level l that are incident to the batch or marked;
 * those with up(v) > (2+3/lambda)(1+delta)^{gn(l)} move to l+1 together.  After
 * the moves, neighbours on level l+1 that now violate Invariant 1 are marked, and a
 * mover stays marked only while it still violates Invariant 1 at l+1.
 * bucket[l] lists vertices that may be candidates at level l.
 */
static int track_batch(orc_plds *h, int op, const uint64_t *keys, int64_t m);

/* Number of neighbours of v on level x or above (by definition). */
static int32_t count_at_or_above(const orc_plds *h, int32_t v, int32_t x) {
    int32_t c = 0;
    for (int32_t j = 0; j < h->deg[v]; ++j) c += h->level[h->nbr[v][j]] >= x;
    return c;
}

/* ORC_JUMP: the target of a violator v of level l -- the smallest x > l with
   count_at_or_above(v, x) <= upmax[gn(x)] on the current levels.  The count does not
   rise and the bound does not fall as x grows, so the test is false below the answer
   and true from it on; the top level passes (its bound is n), and bisection finds
   the first x that passes. */
static int32_t jump_target(const orc_plds *h, int32_t v, int32_t l) {
    int32_t lo = l + 1, hi = h->T.K - 1;
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (count_at_or_above(h, v, mid) <= h->T.upmax[gn(h, mid)]) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

int orc_insert(orc_plds *h, const int32_t *edges, int64_t B) {
    reset_stats(h);
    uint64_t *keys = NULL;
    int64_t m = preprocess(h, edges, B, 0, &keys);
    if (m < 0) return (int)m;
    if (track_batch(h, 0, keys, m)) { free(keys); return ORC_ENOMEM; }
    const int32_t K = h->T.K;
    int rc = ORC_OK;
    int32_t *start_level = NULL;
    ivec *bucket = (ivec *)calloc((size_t)K + 1, sizeof(ivec));
    ivec touched = {0}, movers = {0};
    if (!bucket) { free(keys); return ORC_ENOMEM; }
    /* Algorithm 2: insert every edge of the batch into the graph */
    for (int64_t i = 0; i < m; ++i) {
        int32_t u = (int32_t)(keys[i] >> 32), v = (int32_t)(keys[i] & 0xFFFFFFFFu);
        if (nbr_push(h, u, v) || nbr_push(h, v, u)) { rc = ORC_ENOMEM; goto done; }
        if (!h->incident[u]) { h->incident[u] = 1; iv_push(&touched, u); }
        if (!h->incident[v]) { h->incident[v] = 1; iv_push(&touched, v); }
    }
    start_level = (int32_t *)malloc(sizeof(int32_t) * (touched.len + 1));
    for (int32_t i = 0; i < touched.len; ++i) {
        int32_t v = touched.a[i];
        start_level[i] = h->level[v];
        if (iv_push(&bucket[h->level[v]], v)) { rc = ORC_ENOMEM; goto done; }
    }
    for (int32_t l = 0; l < K; ++l) {
        if (bucket[l].len == 0) continue;
        int32_t s = next_stamp(h);
        movers.len = 0;
        /* the ParFor over candidates on level l that violate Invariant 1 */
        for (int32_t i = 0; i < bucket[l].len; ++i) {
            int32_t v = bucket[l].a[i];
            if (h->stamp[v] == s) continue;
            h->stamp[v] = s;
            if (h->level[v] != l || !(h->incident[v] || h->marked[v])) continue;
            if (up_of(h, v) > h->T.upmax[gn(h, l)]) iv_push(&movers, v);
        }
        free(bucket[l].a);
        bucket[l].a = NULL;
        bucket[l].len = bucket[l].cap = 0;
        if (movers.len == 0) continue;
        if (l + 1 >= K) { rc = ORC_EINTERNAL; goto done; } /* top group can never be violated */
        h->st_rounds++;
        if (h->jump) {
            /* targets on the pre-round levels (the other movers are still on l) */
            int32_t *tgt = (int32_t *)malloc(sizeof(int32_t) * movers.len);
            if (!tgt) { rc = ORC_ENOMEM; goto done; }
            for (int32_t i = 0; i < movers.len; ++i) tgt[i] = jump_target(h, movers.a[i], l);
            for (int32_t i = 0; i < movers.len; ++i) {
                int32_t v = movers.a[i];
                h->level[v] = tgt[i];
                h->marked[v] = 1;
                h->st_moves++;
                h->st_visits += h->deg[v];
            }
            /* a neighbour above l may have gained an up-neighbour: test it on its level */
            int32_t sj = next_stamp(h);
            for (int32_t i = 0; i < movers.len; ++i) {
                int32_t v = movers.a[i];
                for (int32_t j = 0; j < h->deg[v]; ++j) {
                    int32_t w = h->nbr[v][j], lw = h->level[w];
                    if (lw <= l || h->stamp[w] == sj) continue;
                    h->stamp[w] = sj;
                    if (up_of(h, w) > h->T.upmax[gn(h, lw)]) {
                        h->marked[w] = 1;
                        if (iv_push(&bucket[lw], w)) { free(tgt); rc = ORC_ENOMEM; goto done; }
                    }
                }
            }
            /* movers stay candidates on their new level while they violate there */
            for (int32_t i = 0; i < movers.len; ++i) {
                int32_t v = movers.a[i];
                if (up_of(h, v) <= h->T.upmax[gn(h, tgt[i])]) h->marked[v] = 0;
                if (iv_push(&bucket[tgt[i]], v)) { free(tgt); rc = ORC_ENOMEM; goto done; }
            }
            free(tgt);
            continue;
        }
        /* mark and move every violator to level l+1 */
        for (int32_t i = 0; i < movers.len; ++i) {
            int32_t v = movers.a[i];
            h->level[v] = l + 1;
            h->marked[v] = 1;
            h->st_moves++;
            h->st_visits += h->deg[v];
        }
        /* neighbours on level l+1 that now violate Invariant 1 are marked */
        int32_t s2 = next_stamp(h);
        for (int32_t i = 0; i < movers.len; ++i) {
            int32_t v = movers.a[i];
            for (int32_t j = 0; j < h->deg[v]; ++j) {
                int32_t w = h->nbr[v][j];
                if (h->level[w] != l + 1 || h->stamp[w] == s2) continue;
                h->stamp[w] = s2;
                if (up_of(h, w) > h->T.upmax[gn(h, l + 1)]) {
                    h->marked[w] = 1;
                    iv_push(&bucket[l + 1], w);
                }
            }
        }
        /* movers: unmarked when Invariant 1 holds at l+1, otherwise left marked */
        for (int32_t i = 0; i < movers.len; ++i) {
            int32_t v = movers.a[i];
            if (up_of(h, v) <= h->T.upmax[gn(h, l + 1)]) h->marked[v] = 0;
            iv_push(&bucket[l + 1], v);
        }
    }
    for (int32_t i = 0; i < touched.len; ++i) {
        int32_t climbed = h->level[touched.a[i]] - start_level[i];
        if (climbed < 0) h->st_dir_error = 1;
        if (climbed > h->st_max_level_moves) h->st_max_level_moves = climbed;
    }
done:
    /* clear the per-batch flags (marked vertices are always neighbours of movers or movers) */
    for (int32_t i = 0; i < touched.len; ++i) h->incident[touched.a[i]] = 0;
    memset(h->marked, 0, (size_t)h->n);
    for (int32_t l = 0; l <= K; ++l) free(bucket[l].a);
    free(bucket);
    free(touched.a);
    free(movers.a);
    free(start_level);
    free(keys);
    return rc;
}

/*
 * RebalanceDeletions (Algorithm 3).  After removing the batch, every endpoint that
 * violates Invariant 2 gets its desire-level.  Levels l = 0..K-1 are visited in
 * increasing order; all vertices whose desire-level is l move there together; then
 * every neighbour w of a mover with level(w) >= l that violates Invariant 2 on the
 * post-move state has its desire-level recomputed (it always comes out above l).
 */
int orc_delete(orc_plds *h, const int32_t *edges, int64_t B) {
    reset_stats(h);
    uint64_t *keys = NULL;
    int64_t m = preprocess(h, edges, B, 1, &keys);
    if (m < 0) return (int)m;
    if (track_batch(h, 1, keys, m)) { free(keys); return ORC_ENOMEM; }
    const int32_t K = h->T.K;
    int rc = ORC_OK;
    ivec *bucket = (ivec *)calloc((size_t)K + 1, sizeof(ivec));
    ivec touched = {0}, movers = {0};
    int32_t *hist = (int32_t *)malloc(sizeof(int32_t) * ((size_t)K + 2));
    int32_t *moves = (int32_t *)calloc(h->n, sizeof(int32_t));
    if (!bucket || !hist || !moves) { rc = ORC_ENOMEM; goto done; }
    int32_t s = next_stamp(h);
    /* Algorithm 3: remove every edge of the batch from the graph */
    for (int64_t i = 0; i < m; ++i) {
        int32_t u = (int32_t)(keys[i] >> 32), v = (int32_t)(keys[i] & 0xFFFFFFFFu);
        nbr_remove(h, u, v);
        nbr_remove(h, v, u);
        if (h->stamp[u] != s) { h->stamp[u] = s; iv_push(&touched, u); }
        if (h->stamp[v] != s) { h->stamp[v] = s; iv_push(&touched, v); }
    }
    /* vertices whose up*-degree falls below (1+delta)^{gn(level-1)} compute dl */
    for (int32_t i = 0; i < touched.len; ++i) {
        int32_t v = touched.a[i];
        if (!inv2_ok(h, v)) {
            int32_t d = desire_level(h, v, hist);
            h->dl[v] = d;
            iv_push(&bucket[d], v);
        }
    }
    for (int32_t l = 0; l < K; ++l) {
        if (bucket[l].len == 0) continue;
        movers.len = 0;
        int32_t s1 = next_stamp(h);
        for (int32_t i = 0; i < bucket[l].len; ++i) {
            int32_t v = bucket[l].a[i];
            if (h->stamp[v] == s1) continue;
            h->stamp[v] = s1;
            if (h->dl[v] == l) iv_push(&movers, v);
        }
        free(bucket[l].a);
        bucket[l].a = NULL;
        bucket[l].len = bucket[l].cap = 0;
        if (movers.len == 0) continue;
        h->st_rounds++;
        /* move every vertex whose desire-level is l to level l */
        for (int32_t i = 0; i < movers.len; ++i) {
            int32_t v = movers.a[i];
            if (h->level[v] <= l) h->st_dir_error = 1;
            h->level[v] = l;
            h->dl[v] = -1;
            h->st_moves++;
            h->st_visits += h->deg[v];
            if (++moves[v] > h->st_max_level_moves) h->st_max_level_moves = moves[v];
        }
        /* neighbours at or above l that now violate Invariant 2 get dl recomputed */
        int32_t s2 = next_stamp(h);
        for (int32_t i = 0; i < movers.len; ++i) {
            int32_t v = movers.a[i];
            for (int32_t j = 0; j < h->deg[v]; ++j) {
                int32_t w = h->nbr[v][j];
                if (h->level[w] < l || h->stamp[w] == s2) continue;
                h->stamp[w] = s2;
                if (inv2_ok(h, w)) continue;
                int32_t d = desire_level(h, w, hist);
                if (d <= l) { rc = ORC_EINTERNAL; goto done; } /* would contradict the level lemma */
                if (d != h->dl[w]) {
                    h->dl[w] = d;
                    iv_push(&bucket[d], w);
                }
            }
        }
    }
done:
    if (bucket)
        for (int32_t l = 0; l <= K; ++l) free(bucket[l].a);
    free(bucket);
    free(touched.a);
    free(movers.a);
    free(hist);
    free(moves);
    free(keys);
    return rc;
}

/* Update(B) (Algorithm 1): insertions of the batch first, then its deletions. */
int orc_update(orc_plds *h, const int32_t *ins, int64_t nins, const int32_t *del, int64_t ndel) {
    int rc = orc_insert(h, ins, nins);
    if (rc != ORC_OK) return rc;
    return orc_delete(h, del, ndel);
}

/* Coreness estimate (Definition): (1+delta)^{max(floor((level+1)/Lg) - 1, 0)}, 0 when deg = 0. */
int orc_coreness_exponent(const orc_plds *h, int32_t *out) {
    for (int32_t v = 0; v < h->n; ++v) {
        if (h->deg[v] == 0) { out[v] = -1; continue; }
        int32_t g = (h->level[v] + 1) / h->T.Lg - 1;
        out[v] = g > 0 ? g : 0;
    }
    return ORC_OK;
}

int orc_coreness(const orc_plds *h, double *out) {
    double one_plus = 1.0 + (double)h->T.dnum / (double)h->T.dden;
    for (int32_t v = 0; v < h->n; ++v) {
        if (h->deg[v] == 0) { out[v] = 0.0; continue; }
        int32_t g = (h->level[v] + 1) / h->T.Lg - 1;
        if (g < 0) g = 0;
        double x = 1.0;
        for (int32_t i = 0; i < g; ++i) x *= one_plus;
        out[v] = x;
    }
    return ORC_OK;
}

int orc_levels(const orc_plds *h, int32_t *out) {
    memcpy(out, h->level, sizeof(int32_t) * h->n);
    return ORC_OK;
}

/* deg, up, up* of every vertex, each recounted from its definition */
int orc_counters(const orc_plds *h, int32_t *deg, int32_t *up, int32_t *upstar) {
    for (int32_t v = 0; v < h->n; ++v) {
        deg[v] = h->deg[v];
        up[v] = up_of(h, v);
        upstar[v] = upstar_of(h, v);
    }
    return ORC_OK;
}

/* Invariants 1 and 2 for every vertex; deg = 0 => level 0.  Bit 1: Inv-1, 2: Inv-2, 4: isolated. */
int orc_check(const orc_plds *h) {
    int bad = 0;
    for (int32_t v = 0; v < h->n; ++v) {
        if (h->level[v] < 0 || h->level[v] >= h->T.K) return 8;
        if (!inv1_ok(h, v)) bad |= 1;
        if (!inv2_ok(h, v)) bad |= 2;
        if (h->deg[v] == 0 && h->level[v] != 0) bad |= 4;
    }
    return bad;
}

int orc_num_edges(const orc_plds *h, int64_t *m) {
    int64_t s = 0;
    for (int32_t v = 0; v < h->n; ++v) s += h->deg[v];
    *m = s / 2;
    return ORC_OK;
}

/* every edge (u<v) once, in vertex order */
int orc_edges(const orc_plds *h, int32_t *out) {
    int64_t k = 0;
    for (int32_t u = 0; u < h->n; ++u)
        for (int32_t j = 0; j < h->deg[u]; ++j) {
            int32_t v = h->nbr[u][j];
            if (u < v) { out[2 * k] = u; out[2 * k + 1] = v; ++k; }
        }
    return ORC_OK;
}

int orc_stats(const orc_plds *h, int64_t *out /* [12] */) {
    out[0] = h->st_submitted;
    out[1] = h->st_selfloops;
    out[2] = h->st_duplicates;
    out[3] = h->st_filtered;
    out[4] = h->st_valid;
    out[5] = h->st_rounds;
    out[6] = h->st_moves;
    out[7] = h->st_visits;
    out[8] = h->st_dl_evals;
    out[9] = h->st_dl_visits;
    out[10] = h->st_max_level_moves;
    out[11] = h->st_dir_error;
    return ORC_OK;
}

int orc_params(const orc_plds *h, int32_t *out /* [4] t,Lg,G,K */) {
    out[0] = h->T.t;
    out[1] = h->T.Lg;
    out[2] = h->T.G;
    out[3] = h->T.K;
    return ORC_OK;
}

/* Test hooks used to stage the paper's worked examples: set a level, add edges
 * without rebalancing. */
int orc_set_level(orc_plds *h, int32_t v, int32_t l) {
    if (v < 0 || v >= h->n || l < 0 || l >= h->T.K) return ORC_EINVAL;
    h->level[v] = l;
    return ORC_OK;
}

int orc_add_edges_raw(orc_plds *h, const int32_t *edges, int64_t B) {
    for (int64_t i = 0; i < B; ++i) {
        int32_t u = edges[2 * i], v = edges[2 * i + 1];
        if (u < 0 || u >= h->n || v < 0 || v >= h->n || u == v) return ORC_EINVAL;
        if (has_edge(h, u, v)) continue;
        if (nbr_push(h, u, v) || nbr_push(h, v, u)) return ORC_ENOMEM;
    }
    return ORC_OK;
}

/*
 * Exact coreness by Matula-Beck bucket peeling: repeatedly remove a vertex of
 * minimum remaining degree; its coreness is the largest minimum seen so far.
 * Bucket queue over degrees, O(n + m).  edges: m undirected pairs, no duplicates.
 */
int orc_exact_coreness(int32_t n, const int32_t *edges, int64_t m, int32_t *core) {
    int32_t *d = (int32_t *)calloc(n, sizeof(int32_t));
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *adj = (int32_t *)malloc(sizeof(int32_t) * (2 * m + 1));
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
    int32_t *vert = (int32_t *)malloc(sizeof(int32_t) * (n + 1));
    int32_t *bin = NULL;
    int rc = ORC_OK;
    if (!d || !off || !adj || !pos || !vert) { rc = ORC_ENOMEM; goto out; }
    for (int64_t i = 0; i < m; ++i) {
        int32_t u = edges[2 * i], v = edges[2 * i + 1];
        if (u < 0 || u >= n || v < 0 || v >= n || u == v) { rc = ORC_EINVAL; goto out; }
        d[u]++;
        d[v]++;
    }
    for (int32_t v = 0; v < n; ++v) off[v + 1] = off[v] + d[v];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (n + 1));
        memcpy(fill, off, sizeof(int64_t) * (n + 1));
        for (int64_t i = 0; i < m; ++i) {
            int32_t u = edges[2 * i], v = edges[2 * i + 1];
            adj[fill[u]++] = v;
            adj[fill[v]++] = u;
        }
        free(fill);
    }
    int32_t maxd = 0;
    for (int32_t v = 0; v < n; ++v) if (d[v] > maxd) maxd = d[v];
    bin = (int32_t *)calloc((size_t)maxd + 2, sizeof(int32_t));
    for (int32_t v = 0; v < n; ++v) bin[d[v]]++;
    int32_t start = 0;
    for (int32_t k = 0; k <= maxd; ++k) { int32_t c = bin[k]; bin[k] = start; start += c; }
    for (int32_t v = 0; v < n; ++v) { pos[v] = bin[d[v]]; vert[pos[v]] = v; bin[d[v]]++; }
    for (int32_t k = maxd; k >= 1; --k) bin[k] = bin[k - 1];
    bin[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t v = vert[i];
        for (int64_t j = off[v]; j < off[v + 1]; ++j) {
            int32_t u = adj[j];
            if (d[u] > d[v]) {
                int32_t du = d[u], pu = pos[u], pw = bin[du], w = vert[pw];
                if (u != w) { pos[u] = pw; vert[pu] = w; pos[w] = pu; vert[pw] = u; }
                bin[du]++;
                d[u]--;
            }
        }
    }
    for (int32_t v = 0; v < n; ++v) core[v] = d[v];
out:
    free(d);
    free(off);
    free(adj);
    free(pos);
    free(vert);
    free(bin);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Low out-degree orientation (Section "O(alpha) Out-Degree Orientation",    */
/* Algorithm 5).                                                             */
/* An edge goes from the endpoint on the lower level to the one on the       */
/* higher level; on equal levels from the lower id to the higher id (the     */
/* reading of Algorithm 5's flip conditions; the section's prose says the    */
/* opposite, see the design notes).                                          */
/* ------------------------------------------------------------------------- */

/* 1 if the edge {u, v} goes from u to v under the level array lv */
static int goes_from(const int32_t *lv, int32_t u, int32_t v) {
    return lv[u] < lv[v] || (lv[u] == lv[v] && u < v);
}

/* Keep (1) or stop keeping (0) what orc_flips and orc_oriented_updates need. */
int orc_track(orc_plds *h, int on) {
    h->track = on ? 1 : 0;
    return ORC_OK;
}

static int track_batch(orc_plds *h, int op, const uint64_t *keys, int64_t m) {
    if (!h->track) return 0;
    if (!h->old_level && !(h->old_level = (int32_t *)malloc(sizeof(int32_t) * h->n))) return -1;
    memcpy(h->old_level, h->level, sizeof(int32_t) * h->n);
    free(h->last_keys);
    h->last_keys = (uint64_t *)malloc(sizeof(uint64_t) * (m > 0 ? m : 1));
    if (!h->last_keys) return -1;
    if (m > 0) memcpy(h->last_keys, keys, sizeof(uint64_t) * m);
    h->last_m = m;
    h->last_op = op;
    return 0;
}

/* tail[i] = the endpoint edge i is oriented from, -1 if the edge is absent or an id
   is out of range */
int orc_orient(const orc_plds *h, const int32_t *edges, int64_t B, int32_t *tail) {
    for (int64_t i = 0; i < B; ++i) {
        int32_t u = edges[2 * i], v = edges[2 * i + 1];
        if (u < 0 || v < 0 || u >= h->n || v >= h->n || u == v || !has_edge(h, u, v)) {
            tail[i] = -1;
            continue;
        }
        tail[i] = goes_from(h->level, u, v) ? u : v;
    }
    return ORC_OK;
}

/* out[v] = number of edges oriented away from v */
int orc_out_degrees(const orc_plds *h, int32_t *out) {
    for (int32_t v = 0; v < h->n; ++v) {
        int32_t c = 0;
        for (int32_t j = 0; j < h->deg[v]; ++j) c += goes_from(h->level, v, h->nbr[v][j]);
        out[v] = c;
    }
    return ORC_OK;
}

static int in_sorted(const uint64_t *a, int64_t n, uint64_t k) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] == k) return 1;
        if (a[mid] < k) lo = mid + 1; else hi = mid - 1;
    }
    return 0;
}

/*
 * F of the last batch: the edges present before and after it whose orientation
 * changed, each as (tail, head) BEFORE the flip, sorted.  Up to cap pairs are
 * written to out; *count gets their total.  Needs orc_track(h, 1) before the batch.
 */
int orc_flips(const orc_plds *h, int32_t *out, int64_t cap, int64_t *count) {
    if (!h->track || h->last_op < 0) return ORC_EINVAL;
    int64_t k = 0;
    uint64_t *acc = NULL;
    int64_t acap = 0;
    for (int32_t u = 0; u < h->n; ++u) {
        for (int32_t j = 0; j < h->deg[u]; ++j) {
            int32_t v = h->nbr[u][j];
            if (v < u) continue; /* each edge once, from its lower endpoint */
            if (h->last_op == 0 && in_sorted(h->last_keys, h->last_m, ekey(u, v))) continue; /* inserted now */
            int before = goes_from(h->old_level, u, v), after = goes_from(h->level, u, v);
            if (before == after) continue;
            if (k == acap) {
                acap = acap ? 2 * acap : 64;
                uint64_t *t = (uint64_t *)realloc(acc, sizeof(uint64_t) * acap);
                if (!t) { free(acc); return ORC_ENOMEM; }
                acc = t;
            }
            acc[k++] = before ? ekey(u, v) : ekey(v, u);
        }
    }
    if (k > 1) qsort(acc, (size_t)k, sizeof(uint64_t), cmp_u64);
    for (int64_t i = 0; i < k && i < cap; ++i) {
        out[2 * i] = (int32_t)(acc[i] >> 32);
        out[2 * i + 1] = (int32_t)(acc[i] & 0xFFFFFFFFu);
    }
    *count = k;
    free(acc);
    return ORC_OK;
}

/*
 * J of the last batch: its valid updates as (tail, head), insertions oriented after
 * the batch, deletions before it (Algorithm 5), sorted.
 */
int orc_oriented_updates(const orc_plds *h, int32_t *out, int64_t cap, int64_t *count) {
    if (!h->track || h->last_op < 0) return ORC_EINVAL;
    const int32_t *lv = h->last_op == 0 ? h->level : h->old_level;
    uint64_t *acc = (uint64_t *)malloc(sizeof(uint64_t) * (h->last_m > 0 ? h->last_m : 1));
    if (!acc) return ORC_ENOMEM;
    for (int64_t i = 0; i < h->last_m; ++i) {
        int32_t u = (int32_t)(h->last_keys[i] >> 32), v = (int32_t)(h->last_keys[i] & 0xFFFFFFFFu);
        acc[i] = goes_from(lv, u, v) ? ekey(u, v) : ekey(v, u);
    }
    if (h->last_m > 1) qsort(acc, (size_t)h->last_m, sizeof(uint64_t), cmp_u64);
    for (int64_t i = 0; i < h->last_m && i < cap; ++i) {
        out[2 * i] = (int32_t)(acc[i] >> 32);
        out[2 * i + 1] = (int32_t)(acc[i] & 0xFFFFFFFFu);
    }
    *count = h->last_m;
    free(acc);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Static (2+eps')-approximate k-core (Section "Static (2+eps)-Approximate    */
/* k-Core", Algorithm 6): bucketed peeling with thresholds (1+eps)^b.         */
/*                                                                           */
/* Readings (listed in the design notes):                                    */
/*  - eps = (sqrt(4 eps' + 9) - 3) / 2 (so (2+eps)(1+eps) = 2 + eps'),       */
/*    delta = 2 / eps, in double; thresholds thr[b] = (1+eps)^b by repeated  */
/*    multiplication from thr[0] = 1; bucket(C) = the smallest b with        */
/*    thr[b] >= C, i.e. ceil(log_{1+eps} C) decided by comparisons.          */
/*  - a vertex's estimate is thr[its bucket when peeled] (the worked         */
/*    example's values); isolated vertices get 0 and are never peeled.      */
/*  - the outer loop sets t to the lowest non-empty bucket; up to            */
/*    J = ceil(log_{1+delta} n) inner iterations each peel the whole lowest  */
/*    bucket, then update every surviving neighbour:                         */
/*    C = max(C - r, ceil((1+eps)^(t-1))), bucket = max(bucket(C), t); the   */
/*    next inner iteration runs while thr[next lowest bucket] <=             */
/*    (2+eps) thr[t].                                                        */
/* ------------------------------------------------------------------------- */
#define ORC_MAX_BUCKETS 4096

/* The threshold table and the loop constants; 0 on success. */
static int static_params(int32_t n, double eps_prime, double *thr, int32_t *nb, int32_t *J, double *eps_out) {
    if (!(eps_prime > 0.0) || n < 1) return -1;
    double eps = (sqrt(4.0 * eps_prime + 9.0) - 3.0) / 2.0;
    if (!(eps > 0.0)) return -1;
    double delta = 2.0 / eps;
    /* J = ceil(log_{1+delta} n): the smallest J >= 1 with (1+delta)^J >= n */
    int32_t j = 1;
    double p = 1.0 + delta;
    while (p < (double)n && j < 100000) { p *= 1.0 + delta; ++j; }
    /* thresholds up to the first one >= n (no degree exceeds n - 1) */
    int32_t b = 0;
    thr[0] = 1.0;
    while (thr[b] < (double)n) {
        if (b + 1 >= ORC_MAX_BUCKETS) return -1;
        thr[b + 1] = thr[b] * (1.0 + eps);
        ++b;
    }
    *nb = b + 1;
    *J = j;
    *eps_out = eps;
    return 0;
}

static int32_t bucket_of(const double *thr, int32_t nb, int32_t c) {
    int32_t b = 0;
    while (b < nb - 1 && thr[b] < (double)c) ++b;
    return b;
}

/*
 * est[v] for the current graph of h; stats[0] = outer iterations, stats[1] = inner
 * iterations (peeled buckets), stats[2] = neighbour visits (may be NULL).
 */
int orc_static_coreness(const orc_plds *h, double eps_prime, double *est, int64_t *stats) {
    const int32_t n = h->n;
    static double thr[ORC_MAX_BUCKETS];
    int32_t nb = 0, J = 0;
    double eps = 0.0;
    if (static_params(n, eps_prime, thr, &nb, &J, &eps)) return ORC_EINVAL;
    int32_t *C = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *bk = (int32_t *)malloc(sizeof(int32_t) * n);
    int32_t *r = (int32_t *)calloc(n, sizeof(int32_t));
    uint8_t *alive = (uint8_t *)calloc(n, 1), *inI = (uint8_t *)calloc(n, 1);
    if (!C || !bk || !r || !alive || !inI) {
        free(C); free(bk); free(r); free(alive); free(inI);
        return ORC_ENOMEM;
    }
    int64_t left = 0, outer = 0, inner = 0, visits = 0;
    for (int32_t v = 0; v < n; ++v) {
        est[v] = 0.0;
        C[v] = h->deg[v];
        if (C[v] > 0) {
            alive[v] = 1;
            bk[v] = bucket_of(thr, nb, C[v]);
            ++left;
        }
    }
    while (left > 0) {
        int32_t bkt = nb;
        for (int32_t v = 0; v < n; ++v)
            if (alive[v] && bk[v] < bkt) bkt = bk[v];
        const int32_t t = bkt;
        ++outer;
        /* ceil((1+eps)^(t-1)): 1 for t = 0 */
        const int32_t floor_c = t == 0 ? 1 : (int32_t)ceil(thr[t - 1]);
        for (int32_t j = 0; j < J; ++j) {
            ++inner;
            /* I: the whole bucket bkt */
            for (int32_t v = 0; v < n; ++v)
                if (alive[v] && bk[v] == bkt) {
                    inI[v] = 1;
                    alive[v] = 0;
                    est[v] = thr[bkt];
                    --left;
                }
            /* R: r_v = neighbours of v in I, for surviving v */
            for (int32_t u = 0; u < n; ++u) {
                if (!inI[u]) continue;
                for (int32_t k = 0; k < h->deg[u]; ++k) {
                    int32_t v = h->nbr[u][k];
                    ++visits;
                    if (alive[v]) r[v]++;
                }
            }
            for (int32_t v = 0; v < n; ++v) {
                inI[v] = 0;
                if (!r[v]) continue;
                int32_t c = C[v] - r[v];
                C[v] = c > floor_c ? c : floor_c;
                int32_t nbk = bucket_of(thr, nb, C[v]);
                bk[v] = nbk > t ? nbk : t;
                r[v] = 0;
            }
            if (left == 0) break;
            int32_t next = nb;
            for (int32_t v = 0; v < n; ++v)
                if (alive[v] && bk[v] < next) next = bk[v];
            if (thr[next] <= (2.0 + eps) * thr[t]) bkt = next;
            else break;
        }
    }
    if (stats) { stats[0] = outer; stats[1] = inner; stats[2] = visits; }
    free(C); free(bk); free(r); free(alive); free(inI);
    return ORC_OK;
}

/* The threshold table (for the tests): up to cap entries; returns the count. */
int32_t orc_static_thresholds(int32_t n, double eps_prime, double *thr_out, int32_t cap, int32_t *J) {
    static double thr[ORC_MAX_BUCKETS];
    int32_t nb = 0;
    double eps = 0.0;
    if (static_params(n, eps_prime, thr, &nb, J, &eps)) return ORC_EINVAL;
    for (int32_t i = 0; i < nb && i < cap; ++i) thr_out[i] = thr[i];
    return nb;
}
