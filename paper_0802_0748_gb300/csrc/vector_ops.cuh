// Deterministic reductions of the standalone vector kernels (256-thread
// blocks) of the ground-state iteration.
#pragma once
#include "common.cuh"

namespace scocg {

// Reductions of the standalone vector kernels (256-thread blocks): a block's
// partial sum lands in part[blockIdx.x]; every consuming block adds the G
// partials in the same fixed order, so all blocks see the same bit-identical
// total without a separate reduction launch.
constexpr int kVecBlock = 256;

__device__ __forceinline__ void block_partial(double v, double* part) {
    __shared__ double s_w[kVecBlock / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kVecBlock / 32; ++w) t += s_w[w];
        part[blockIdx.x] = t;
    }
}

__device__ __forceinline__ double sum_partials(const double* part, int G) {
    __shared__ double s_w[kVecBlock / 32];
    __shared__ double s_tot;
    double v = 0.0;
    for (int c = threadIdx.x; c < G; c += kVecBlock) v += __ldcg(part + c);
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kVecBlock / 32; ++w) t += s_w[w];
        s_tot = t;
    }
    __syncthreads();
    return s_tot;
}

}  // namespace scocg
