// Bit-string basis of a fixed-popcount sector (shared by the Hubbard models):
// a string's rank is its position among all strings of the same popcount in
// ascending order, which is the combinatorial number system sum_j C(pos_j, j + 1)
// over its set bits pos_0 < pos_1 < ...
#pragma once
#include <stdint.h>

namespace scocg {

__host__ __device__ inline int64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

__device__ inline int64_t rank_of(uint32_t s) {
    int64_t r = 0;
    int j = 0;
    for (int pos = 0; pos < 32; ++pos)
        if ((s >> pos) & 1u) { ++j; r += binom(pos, j); }
    return r;
}

__device__ inline uint32_t unrank(int64_t r, int k, int L) {
    uint32_t s = 0;
    for (int j = k; j >= 1; --j) {
        int p = j - 1;
        while (p + 1 < L && binom(p + 1, j) <= r) ++p;
        s |= 1u << p;
        r -= binom(p, j);
    }
    return s;
}

}  // namespace scocg
