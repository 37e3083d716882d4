// Exact integer thresholds of the PLDS (host side of the CUDA library).
//
// Invariant 1 (Section "Detailed PLDS Algorithm"): a vertex on a level of group i
// has at most (2+3/lambda)(1+delta)^i up-neighbours; Invariant 2: a vertex on
// level l > 0 with l-1 in group i has at least (1+delta)^i up*-neighbours.  Since
// degrees are integers the tests become up > floor(c(1+delta)^i) and
// up* < ceil((1+delta)^i).  Both are computed exactly from delta = p/q and
// lambda = a/b (denominator 10^6) with arbitrary-precision integers and binary
// long division, and clamped to n (no degree reaches n).
#include "plds_tables.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

namespace pl {
namespace {

// Non-negative integer, base 2^32 limbs, least significant first, no leading zeros.
struct Nat {
    std::vector<uint32_t> w;
    static Nat of(uint64_t v) {
        Nat r;
        while (v) { r.w.push_back((uint32_t)v); v >>= 32; }
        return r;
    }
    size_t bits() const {
        if (w.empty()) return 0;
        uint32_t top = w.back();
        size_t b = 0;
        while (top) { ++b; top >>= 1; }
        return (w.size() - 1) * 32 + b;
    }
    void trim() { while (!w.empty() && w.back() == 0) w.pop_back(); }
};

Nat mul(const Nat &a, uint32_t m) {
    Nat r;
    uint64_t carry = 0;
    for (uint32_t x : a.w) {
        uint64_t t = (uint64_t)x * m + carry;
        r.w.push_back((uint32_t)t);
        carry = t >> 32;
    }
    if (carry) r.w.push_back((uint32_t)carry);
    r.trim();
    return r;
}

Nat shl(const Nat &a, size_t s) {
    Nat r;
    size_t limbs = s / 32, bits = s % 32;
    r.w.assign(limbs, 0);
    uint32_t carry = 0;
    for (uint32_t x : a.w) {
        r.w.push_back(bits ? (x << bits) | carry : x);
        carry = bits ? x >> (32 - bits) : 0;
    }
    if (carry) r.w.push_back(carry);
    r.trim();
    return r;
}

int cmp(const Nat &a, const Nat &b) {
    if (a.w.size() != b.w.size()) return a.w.size() < b.w.size() ? -1 : 1;
    for (size_t i = a.w.size(); i-- > 0;)
        if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
    return 0;
}

void sub_in(Nat &a, const Nat &b) {  // a -= b, a >= b
    int64_t borrow = 0;
    for (size_t i = 0; i < a.w.size(); ++i) {
        int64_t t = (int64_t)a.w[i] - (i < b.w.size() ? b.w[i] : 0) - borrow;
        borrow = t < 0;
        a.w[i] = (uint32_t)(t + (borrow ? (int64_t)1 << 32 : 0));
    }
    a.trim();
}

// floor(x / y) and whether the division was exact, for quotients below 2^31.
int64_t divide(const Nat &x, const Nat &y, bool *exact) {
    Nat r = x;
    int64_t q = 0;
    for (int b = 31; b >= 0; --b) {
        Nat ys = shl(y, (size_t)b);
        if (cmp(ys, r) <= 0) {
            sub_in(r, ys);
            q |= (int64_t)1 << b;
        }
    }
    *exact = r.w.empty();
    return q;
}

}  // namespace

int build_tables(int32_t n, double delta, double lambda, int32_t levels_per_group, Tables *out, bool heuristic) {
    if (n < 1 || !(delta > 0) || !(lambda > 0) || delta > 1e6 || lambda > 1e6 || levels_per_group < 0) return -1;
    int64_t p = std::llround(delta * 1e6), q = 1000000, a = std::llround(lambda * 1e6), b = 1000000;
    if (p <= 0 || a <= 0) return -1;
    int64_t g1 = std::gcd(p, q), g2 = std::gcd(a, b);
    p /= g1; q /= g1; a /= g2; b /= g2;
    out->delta_num = p; out->delta_den = q; out->lambda_num = a; out->lambda_den = b;
    // t: smallest t >= 0 with (q+p)^t >= n q^t
    Nat num = Nat::of(1), den = Nat::of(1);
    int t = 0;
    while (cmp(num, mul(den, (uint32_t)n)) < 0) {
        num = mul(num, (uint32_t)(q + p));
        den = mul(den, (uint32_t)q);
        if (++t > kMaxGroupsHost - 1 || num.bits() > 20000) return -1;
    }
    out->t = t;
    out->Lg = levels_per_group > 0 ? levels_per_group : 4 * std::max(1, t);
    out->G = t + 1;
    int64_t K = (int64_t)out->G * out->Lg;
    if (K >= (int64_t)1 << 24) return -1;
    out->K = (int32_t)K;
    out->upmax.assign(out->G, 0);
    out->dnmin.assign(out->G, 0);
    // c = (2a + 3b) / a, or 11/10 for the heuristic ; (1+delta)^i = (q+p)^i / q^i
    const uint32_t cn = heuristic ? 11u : (uint32_t)(2 * a + 3 * b), cd = heuristic ? 10u : (uint32_t)a;
    Nat pw = Nat::of(1), qw = Nat::of(1);
    for (int i = 0; i < out->G; ++i) {
        Nat x = mul(pw, cn);
        Nat y = mul(qw, cd);
        bool exact;
        // clamp: x >= n*y  <=>  floor(x/y) >= n
        if (cmp(x, mul(y, (uint32_t)n)) >= 0) out->upmax[i] = n;
        else out->upmax[i] = (int32_t)divide(x, y, &exact);
        if (cmp(pw, mul(qw, (uint32_t)n)) >= 0) {
            out->dnmin[i] = n;
        } else {
            int64_t f = divide(pw, qw, &exact);
            out->dnmin[i] = (int32_t)std::min<int64_t>(exact ? f : f + 1, n);
        }
        pw = mul(pw, (uint32_t)(q + p));
        qw = mul(qw, (uint32_t)q);
    }
    // (1+delta)^g as doubles for the coreness estimate
    out->pow.assign(out->G, 1.0);
    long double base = 1.0L + (long double)p / (long double)q, acc = 1.0L;
    for (int i = 0; i < out->G; ++i) {
        out->pow[i] = (double)acc;
        acc *= base;
    }
    return 0;
}

int32_t opt_levels_per_group(int64_t m, double delta) {
    if (m < 0 || m > (int64_t)0xffffffffLL || !(delta > 0) || delta > 1e6) return -1;
    int64_t p = std::llround(delta * 1e6), q = 1000000;
    if (p <= 0) return -1;
    const int64_t g = std::gcd(p, q);
    p /= g;
    q /= g;
    if (p + q > (int64_t)0xffffffffLL) return -1;
    Nat num = Nat::of(1), den = Nat::of(1);
    for (int32_t L = 1; L <= (1 << 20); ++L) {
        for (int k = 0; k < 50; ++k) {
            num = mul(num, (uint32_t)(p + q));
            den = mul(den, (uint32_t)q);
        }
        if (num.bits() > 20000) return -1;
        if (cmp(num, mul(den, (uint32_t)m)) >= 0) return L;
    }
    return -1;
}

int build_static_tables(int32_t n, double eps_prime, StaticTables *out) {
    if (n < 1 || !(eps_prime > 0) || eps_prime > 1e9) return -1;
    const double eps = (std::sqrt(4.0 * eps_prime + 9.0) - 3.0) / 2.0;
    if (!(eps > 0)) return -1;
    const double delta = 2.0 / eps;
    int32_t J = 1;
    for (double p = 1.0 + delta; p < (double)n && J < 100000; p *= 1.0 + delta) ++J;
    out->thr.assign(1, 1.0);
    while (out->thr.back() < (double)n) {
        if (out->thr.size() >= 4096) return -1;
        out->thr.push_back(out->thr.back() * (1.0 + eps));
    }
    const size_t nb = out->thr.size();
    out->lim.resize(nb);
    out->floor_c.resize(nb);
    for (size_t t = 0; t < nb; ++t) {
        out->lim[t] = (2.0 + eps) * out->thr[t];
        out->floor_c[t] = t == 0 ? 1 : (int32_t)std::ceil(out->thr[t - 1]);
    }
    out->J = J;
    out->eps = eps;
    return 0;
}

}  // namespace pl
