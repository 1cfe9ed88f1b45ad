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

// ---- packed pairs: the real and imaginary parts of a compensated complex
// number go through the same error-free transformations, so the two are
// computed together with the GPU's paired FP32 instructions (one instruction,
// two correctly rounded FP32 results).  Layout of a float4 {re.hi, im.hi,
// re.lo, im.lo}: hi pair (x, y), lo pair (z, w).
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pk_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 pk_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pk_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pk_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 pk4(float2 h, float2 l) { return make_float4(h.x, h.y, l.x, l.y); }

// TwoSum on both lanes: s + e == a + b exactly
__device__ __forceinline__ void pk_two_sum(float2 a, float2 b, float2& s, float2& e) {
    s = pk_add(a, b);
    const float2 bb = pk_sub(s, a);
    e = pk_add(pk_sub(a, pk_sub(s, bb)), pk_sub(b, bb));
}
// Fast2Sum normalisation of both lanes (hi, lo) -> (s, e), |lo| small
__device__ __forceinline__ void pk_norm(float2& hi, float2& lo) {
    const float2 s = pk_add(hi, lo);
    lo = pk_sub(lo, pk_sub(s, hi));
    hi = s;
}
// (ah, al) += (xh + xl) * (yh + yl) lane by lane, the product exact to DF and
// the sum by TwoSum, without renormalising the accumulator
__device__ __forceinline__ void pk_acc_prod(float2& ah, float2& al, float2 xh, float2 xl, float2 yh, float2 yl) {
    const float2 p = pk_mul(xh, yh);
    float2 e = pk_fma(xh, yh, pk_neg(p));
    e = pk_fma(xh, yl, pk_fma(xl, yh, e));
    float2 s, t;
    pk_two_sum(ah, p, s, t);
    ah = s;
    al = pk_add(al, pk_add(t, e));
}

// complex a * b + c: (re, im) += (a.re, a.re) (b.re, b.im) + (-a.im, a.im) (b.im, b.re)
__device__ __forceinline__ float4 vcfma(float4 a, float4 b, float4 c) {
    float2 h = hi2(c), l = lo2(c);
    const float2 bh = hi2(b), bl = lo2(b);
    pk_acc_prod(h, l, make_float2(a.x, a.x), make_float2(a.z, a.z), bh, bl);
    pk_acc_prod(h, l, make_float2(-a.y, a.y), make_float2(-a.w, a.w), make_float2(bh.y, bh.x),
                make_float2(bl.y, bl.x));
    pk_norm(h, l);
    return pk4(h, l);
}
__device__ __forceinline__ float4 vsub(float4 a, float4 b) {
    float2 s, e;
    pk_two_sum(hi2(a), pk_neg(hi2(b)), s, e);
    e = pk_add(e, pk_sub(lo2(a), lo2(b)));
    pk_norm(s, e);
    return pk4(s, e);
}
// acc += v * x (real float v); acc is kept unnormalised until the apply ends
__device__ __forceinline__ void cfma_r(float4& acc, float v, float4 x) {
    const float2 vv = make_float2(v, v);
    float2 h = hi2(acc), l = lo2(acc);
    const float2 xh = hi2(x);
    const float2 p = pk_mul(vv, xh);
    float2 e = pk_fma(vv, xh, pk_neg(p));
    e = pk_fma(vv, lo2(x), e);
    float2 s, t;
    pk_two_sum(h, p, s, t);
    acc = pk4(s, pk_add(l, pk_add(t, e)));
}
// sum of two unnormalised compensated complex accumulators, normalised
__device__ __forceinline__ float4 vadd_acc(float4 a, float4 b) {
    float2 ah = hi2(a), al = lo2(a), bh = hi2(b), bl = lo2(b);
    pk_norm(ah, al);
    pk_norm(bh, bl);
    float2 s, e;
    pk_two_sum(ah, bh, s, e);
    e = pk_add(e, pk_add(al, bl));
    pk_norm(s, e);
    return pk4(s, e);
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
