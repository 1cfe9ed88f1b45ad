// Shared device helpers of the shifted-COCG library: complex arithmetic on
// double2/float2, cache-hinted loads, the watchdog grid barrier and the
// deterministic block / grid reductions used by the persistent solver kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "scocg.h"

namespace scocg {

constexpr int kMaxProj = 32;        // projections per solve (single right-hand side)
constexpr int kBlock = 512;         // threads per CTA of the persistent kernels
constexpr int kWarps = kBlock / 32;

// ---------------------------------------------------------------- complex
__host__ __device__ __forceinline__ double2 c2(double re, double im) { return make_double2(re, im); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return c2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return c2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return c2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return c2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabs_(double2 a) { return hypot(a.x, a.y); }
// a / b with scaling by the larger component of b (Smith's method) so that
// |b| near the limits of the exponent range neither overflows nor underflows.
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    if (fabs(b.x) >= fabs(b.y)) {
        const double r = b.y / b.x, inv = 1.0 / (b.x + b.y * r);
        return c2((a.x + a.y * r) * inv, (a.y - a.x * r) * inv);
    } else {
        const double r = b.x / b.y, inv = 1.0 / (b.x * r + b.y);
        return c2((a.x * r + a.y) * inv, (a.y * r - a.x) * inv);
    }
}
// 1 / b with the same scaling
__host__ __device__ __forceinline__ double2 crecip(double2 b) {
    if (fabs(b.x) >= fabs(b.y)) {
        const double r = b.y / b.x, inv = 1.0 / (b.x + b.y * r);
        return c2(inv, -r * inv);
    } else {
        const double r = b.x / b.y, inv = 1.0 / (b.x * r + b.y);
        return c2(r * inv, -inv);
    }
}
__host__ __device__ __forceinline__ bool cfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

__device__ __forceinline__ float2 f2(float re, float im) { return make_float2(re, im); }

// Vector element of the two precisions: complex128 (double2) or complex64 (float2).
template <typename R> struct Vec;
template <> struct Vec<double> {
    using T = double2;
    __device__ static __forceinline__ T make(double2 a) { return a; }
    __device__ static __forceinline__ double2 wide(T a) { return a; }
};
template <> struct Vec<float> {
    using T = float2;
    __device__ static __forceinline__ T make(double2 a) { return make_float2((float)a.x, (float)a.y); }
    __device__ static __forceinline__ double2 wide(T a) { return make_double2(a.x, a.y); }
};

template <typename T> __device__ __forceinline__ T vzero();
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// acc += v * x for a real value v and a complex x (FMA in the vector's precision)
__device__ __forceinline__ void cfma_r(double2& acc, double v, double2 x) {
    acc.x = fma(v, x.x, acc.x); acc.y = fma(v, x.y, acc.y);
}
__device__ __forceinline__ void cfma_r(float2& acc, float v, float2 x) {
    acc.x = fmaf(v, x.x, acc.x); acc.y = fmaf(v, x.y, acc.y);
}
// complex a * b + c in the vector precision
__device__ __forceinline__ double2 vcfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 vcfma(float2 a, float2 b, float2 c) {
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 vsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// ---------------------------------------------------------------- compensated FP32
}  // namespace scocg
#include "dfloat.cuh"
namespace scocg {

// Precision tag of the compensated mode: vectors of float4 {re.hi, im.hi,
// re.lo, im.lo}, FP32 H values, FP32 arithmetic with error-free transforms.
struct DF {};
template <> struct Vec<DF> {
    using T = float4;
    __device__ static __forceinline__ T make(double2 a) { return df_from(a); }
    __device__ static __forceinline__ double2 wide(T a) { return df_to(a); }
};
// H value type of each precision
template <typename R> struct ValT { using T = R; };
template <> struct ValT<DF> { using T = float; };
// per-thread accumulator type of the dot products
template <typename R> struct Acc { using T = R; };
template <> struct Acc<DF> { using T = dfs; };
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(dfs v) { return (double)v.hi + (double)v.lo; }

// dynamic shared memory array (the host emulation used for CPU debugging of
// the kernel source gives it static storage)
#ifdef SCOCG_HOST_EMULATION
#define SCOCG_DYN_SHARED(T, name) static T name[16384]
#else
#define SCOCG_DYN_SHARED(T, name) extern __shared__ T name[]
#endif

// ---------------------------------------------------------------- loads
// Streaming loads for H (read once per iteration, larger than L2): evict first.
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ double2 ld_stream(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ int ld_stream(const int* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ double ld_stream(const double* p) { return __ldcs(p); }
// Vector loads that must see other CTAs' writes from earlier phases of the same
// launch: cache at L2 only (never a stale L1 line).
__device__ __forceinline__ double2 ld_l2(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ld_l2(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double ld_l2(const double* p) { return __ldcg(p); }

#ifndef SCOCG_HOST_EMULATION
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
#endif

// ---------------------------------------------------------------- barrier
// Barrier over the `nctas` co-resident CTAs of one solve (the whole grid, or
// one system's share of a multi-system launch).  `count` only ever grows:
// barrier number b completes when it reaches (b + 1) * nctas.  The
// wait gives up after `timeout_ns`, records SCOCG_ERR_TIMEOUT in *status and
// returns false; it also returns false as soon as any CTA has recorded an
// error, so that every CTA leaves the kernel instead of waiting.
struct GridSync {
    unsigned long long* count;
    int* status;
    uint64_t timeout_ns;
    int nctas;
};

__device__ __forceinline__ bool grid_barrier(const GridSync& g, unsigned long long& epoch,
                                             bool skip_arrival = false) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ++epoch;
        const unsigned long long target = epoch * (unsigned long long)g.nctas;
        __threadfence();
        if (!skip_arrival) atomicAdd(g.count, 1ull);
        int ok = 1;
        const uint64_t t0 = globaltimer_ns();
        while (ld_acquire_u64(g.count) < target) {
            if (ld_volatile_i32(g.status) < 0) { ok = 0; break; }
            if (globaltimer_ns() - t0 > g.timeout_ns) {
                atomicCAS(g.status, 0, (int)SCOCG_ERR_TIMEOUT);
                atomicCAS(g.status, 1, (int)SCOCG_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        if (ok && ld_volatile_i32(g.status) < 0) ok = 0;
        __threadfence();   // acquire side: later loads of this CTA see the other CTAs' writes
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void set_error(int* status, int code) {
    int old = atomicCAS(status, 0, code);
    if (old == 1) atomicCAS(status, 1, code);
}

// ---------------------------------------------------------------- checked build
// With -DSCOCG_CHECKED every data-dependent index is tested before use: a bad
// one is recorded in dbg[0..3] = (1, site, index, limit) and the access is
// skipped.  Without it the test compiles away.
#ifdef SCOCG_CHECKED
__device__ __forceinline__ bool chk(unsigned long long* dbg, int site, long long idx, long long lim) {
    if (idx >= 0 && idx < lim) return true;
    if (dbg && atomicCAS(dbg, 0ull, 1ull) == 0ull) {
        dbg[1] = (unsigned long long)site; dbg[2] = (unsigned long long)idx; dbg[3] = (unsigned long long)lim;
    }
    return false;
}
#else
__device__ __forceinline__ bool chk(unsigned long long*, int, long long, long long) { return true; }
#endif

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum `nval` per-thread doubles over the CTA; the result lands in out[0..nval)
// (shared memory) and is visible to all threads after the call.  `scratch`
// must hold kWarps * nval doubles.
__device__ __forceinline__ void block_sum(const double* vals, int nval, double* scratch, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < nval; ++j) {
        double v = warp_sum(vals[j]);
        if (lane == 0) scratch[warp * nval + j] = v;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nval; j += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += scratch[w * nval + j];
        out[j] = s;
    }
    __syncthreads();
}

// Deterministic grid reduction of per-CTA partials part[cta * stride + j],
// j < nval: every CTA computes bit-identical sums (same data, same order).
// The loads of a lane are issued together (up to 16 per lane, grids up to 512
// CTAs in one round) so that the reduction costs one L2 round trip.
// The same sum over value-major partials part[j * G + cta]: a warp's load of
// 32 consecutive CTAs is one coalesced request, and the CTAs' reads after a
// barrier touch G / 32 lines per value instead of G.  Same summation order.
__device__ __forceinline__ void grid_sum_vm1(const double* part, int nval, double* out, int G) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = warp; j < nval; j += kWarps) {
        const double* pj = part + (size_t)j * G;
        double s = 0.0;
        for (int c0 = 0; c0 < G; c0 += 32 * 16) {
            double v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int c = c0 + lane + 32 * u;
                v[u] = c < G ? __ldcg(pj + c) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) s += v[u];
        }
        s = warp_sum(s);
        if (lane == 0) out[j] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ void grid_sum(const double* part, int stride, int nval, double* out, int G) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = warp; j < nval; j += kWarps) {
        double s = 0.0;
        for (int c0 = 0; c0 < G; c0 += 32 * 16) {
            double v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int c = c0 + lane + 32 * u;
                v[u] = c < G ? __ldcg(part + (size_t)c * stride + j) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) s += v[u];
        }
        s = warp_sum(s);
        if (lane == 0) out[j] = s;
    }
    __syncthreads();
}

}  // namespace scocg
