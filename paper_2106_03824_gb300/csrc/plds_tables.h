// Exact per-group thresholds of the PLDS (host side of the CUDA library).
#pragma once
#include <cstdint>
#include <vector>

namespace pl {

constexpr int kMaxGroupsHost = 512;

struct Tables {
    int64_t delta_num, delta_den, lambda_num, lambda_den;
    int32_t t, Lg, G, K;
    std::vector<int32_t> upmax;  // floor((2+3/lambda)(1+delta)^i), clamped to n
    std::vector<int32_t> dnmin;  // ceil((1+delta)^i), clamped to n
    std::vector<double> pow;     // (1+delta)^i
};

// 0 on success, -1 on invalid parameters (n < 1, delta/lambda not positive,
// more than 512 groups or 2^24 levels).
// heuristic: Invariant 1's coefficient 2 + 3/lambda replaced by 1.1.
int build_tables(int32_t n, double delta, double lambda, int32_t levels_per_group, Tables *out,
                 bool heuristic = false);

// Levels per group of the optimised variant: ceil(log_{1+delta}(m) / 50), at least 1
// (the smallest L >= 1 with (1+delta)^(50 L) >= m, exact).  -1 on invalid input
// (m outside [0, 2^32), delta not positive, or powers beyond 20000 bits).
int32_t opt_levels_per_group(int64_t m, double delta);

// Constants of the static approximate k-core (Algorithm 6) for n vertices:
// eps = (sqrt(4 eps' + 9) - 3) / 2, delta = 2 / eps; thr[b] = (1+eps)^b by repeated
// multiplication up to the first value >= n; floor_c[t] = ceil((1+eps)^(t-1)) (1 for
// t = 0); lim[t] = (2+eps) thr[t]; J = ceil(log_{1+delta} n).  -1 on invalid input.
struct StaticTables {
    std::vector<double> thr, lim;
    std::vector<int32_t> floor_c;
    int32_t J = 0;
    double eps = 0;
};
int build_static_tables(int32_t n, double eps_prime, StaticTables *out);

}  // namespace pl
