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
int build_tables(int32_t n, double delta, double lambda, int32_t levels_per_group, Tables *out);

}  // namespace pl
