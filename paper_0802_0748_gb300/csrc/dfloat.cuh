// Compensated FP32 ("double-float") arithmetic for the SCOCG_MIXED_DF mode.
//
// A real number is an unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2
// after normalisation), giving about 44 significant bits with FP32 operations
// only.  The building blocks are the classical error-free transformations:
// TwoSum (Knuth: s + e == a + b exactly), Fast2Sum (Dekker, |a| >= |b|) and
// TwoProd through a fused multiply-add (p + e == a * b exactly).
//
// A complex vector entry is a float4 {re.hi, im.hi, re.lo, im.lo}.
#pragma once
#include <cuda_runtime.h>

namespace scocg {

struct dfs {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = a * b;
    e = fmaf(a, b, -p);
}

__device__ __forceinline__ dfs df_norm(float hi, float lo) {
    dfs r;
    fast_two_sum(hi, lo, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ dfs df_add(dfs a, dfs b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    return df_norm(s, e);
}
__device__ __forceinline__ dfs df_neg(dfs a) { return dfs{-a.hi, -a.lo}; }
__device__ __forceinline__ dfs df_mul(dfs a, dfs b) {
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return df_norm(p, e);
}
// Accumulate the exact-to-DF product a * b into (acc.hi, acc.lo) without
// renormalising acc (normalise once at the end with df_norm).
__device__ __forceinline__ void df_acc_prod(dfs& acc, dfs a, dfs b) {
    float p, e, s, t;
    two_prod(a.hi, b.hi, p, e);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    two_sum(acc.hi, p, s, t);
    acc.hi = s;
    acc.lo += t + e;
}
// acc += v * x for a float v and a DF x (the H apply)
__device__ __forceinline__ void df_acc_fx(dfs& acc, float v, float xhi, float xlo) {
    float p, e, s, t;
    two_prod(v, xhi, p, e);
    e = fmaf(v, xlo, e);
    two_sum(acc.hi, p, s, t);
    acc.hi = s;
    acc.lo += t + e;
}

__device__ __forceinline__ dfs cre(float4 v) { return dfs{v.x, v.z}; }
__device__ __forceinline__ dfs cim(float4 v) { return dfs{v.y, v.w}; }
__device__ __forceinline__ float4 cpack(dfs re, dfs im) { return make_float4(re.hi, im.hi, re.lo, im.lo); }

// complex a * b + c
__device__ __forceinline__ float4 vcfma(float4 a, float4 b, float4 c) {
    dfs re = cre(c), im = cim(c);
    df_acc_prod(re, cre(a), cre(b));
    df_acc_prod(re, df_neg(cim(a)), cim(b));
    df_acc_prod(im, cre(a), cim(b));
    df_acc_prod(im, cim(a), cre(b));
    return cpack(df_norm(re.hi, re.lo), df_norm(im.hi, im.lo));
}
__device__ __forceinline__ float4 vsub(float4 a, float4 b) {
    return cpack(df_add(cre(a), df_neg(cre(b))), df_add(cim(a), df_neg(cim(b))));
}
// acc += v * x (real float v); acc is kept unnormalised until the apply ends
__device__ __forceinline__ void cfma_r(float4& acc, float v, float4 x) {
    dfs re = cre(acc), im = cim(acc);
    df_acc_fx(re, v, x.x, x.z);
    df_acc_fx(im, v, x.y, x.w);
    acc = cpack(re, im);
}

// DF <-> double conversions (FP64 arithmetic: only for scalars and set-up)
__host__ __device__ __forceinline__ float4 df_from(double2 a) {
    const float rh = (float)a.x, ih = (float)a.y;
    return make_float4(rh, ih, (float)(a.x - (double)rh), (float)(a.y - (double)ih));
}
__host__ __device__ __forceinline__ double2 df_to(float4 v) {
    return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}
__device__ __forceinline__ double df_to(dfs v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ dfs warp_sum(dfs v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dfs w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}

}  // namespace scocg
