// Persistent single-right-hand-side shifted-COCG kernel (Sec. III.C of
// arXiv:0802.0748), templated on the vector precision R (double: complex128,
// float: complex64 with FP64 scalars) and on the H-apply functor.
//
// One cooperative launch runs the whole solve.  Each CTA owns a fixed range of
// rows (the apply's "units") and a fixed subset of shifts (k = cta + j*grid).
// Per seed iteration n (matrix A = z_s I - H):
//   phase A  q_n = A r_n + beta_{n-1} q_{n-1}, partial r_n^T q_n      -> barrier
//   phase B  alpha_n = rho_n / (r_n^T q_n) (every CTA, same reduction order);
//            r_{n+1} = r_n - alpha_n q_n; partial r^T r, ||r||^2, c_m^T r -> barrier
//   phase C  rho_{n+1}, beta_n; every CTA updates its own shifts:
//            pi^k_{n+1} = (1 + alpha_n sigma_k) pi^k_n
//                         + (alpha_n beta_{n-1}/alpha_{n-1}) (pi^k_n - pi^k_{n-1}),
//            projected p^k and x^k:  P^k_m = c_m^T r_n / pi^k_n + beta^k_{n-1} P^k_m,
//            X^k_m += alpha^k_n P^k_m, residual ||r_{n+1}|| / (|pi^k_{n+1}| ||b||).
// q_n = A p_n replaces the seed direction p_n (p is never stored); r_n^T q_n
// equals p_n^T A p_n because successive directions are A-conjugate in the
// bilinear form.  When the seed converges first, the unconverged shift with
// the largest residual becomes the new seed (seed switching) with
//   r' = r_{n+1} / pi'_{n+1},  q' = (r_n / pi'_n - r_{n+1} / pi'_{n+1}) / alpha'_n,
// pi^k <- pi^k / pi', sigma_k <- z_k - z_s'.
// MIXED precision additionally carries the seed's p and x (x compensated) and
// every `replace_every` iterations replaces r by the FP64 true residual
// b - A x (reliable update).
#pragma once
#include "common.cuh"

namespace scocg {

constexpr int kMaxProjB = 4;   // unit projections per right-hand side of a block (multi-rhs) solve
#ifndef SCOCG_BSR4_GROUP
#define SCOCG_BSR4_GROUP 4     // slots of the blocked apply whose loads are issued together
#endif
constexpr int kPartC = 10;   // active, best |pi|, arg, bad, pi_prev, pi_cur, alpha_k of arg

struct ShiftState {          // device arrays, [K] or [K][M]
    double2* pi_prev;
    double2* pi_cur;
    double2* sigma;
    double2* alpha_k;        // alpha^k_n of the last update (needed by a switch)
    double2* inv_cur;        // 1 / pi^k_n
    double2* P;              // [K][M] c_m^T p^k
    double2* X;              // [K][M] c_m^T x^k
    int* frozen;
    int* iters;
    double* resid;           // squared residual estimate (||r_k|| / ||b||)^2
};

// What a solve that stopped at max_iter leaves for a later launch to continue
// from (scocg_solve_resume): it stops between the apply of iteration n and
// its first reduction, so the workspace holds r_n, q_n and every shift's
// recurrence after iteration n - 1; these are the seed scalars of that point.
struct ResumeState {       // device, written by CTA 0
    int valid;             // 1: the last solve stopped at max_iter
    int n, seed, n_switch, n_replace, replace_on;
    int rotated;           // the stopping apply visited its units in the rotated order
    int pad;
    double2 alpha_prev, beta_prev, rho, rho_prev, zs;
    double rnorm, bnorm;
    double2 cr_cur[kMaxProj];
};

struct SolveStats {          // device, written by CTA 0
    int status;
    int iters;
    int n_switch;
    int seed;
    int n_replace;
    int pad;
    long long shift_iters;
};

// ---------------------------------------------------------------- applies
// How the persistent kernel's phase A hands units to warps: a contiguous
// range per CTA (the blocked and CSR applies: measured fastest), or unit
// cta + G * (warp + W * j), all CTAs interleaved (the Hubbard apply, whose
// units are up-spin blocks of very different cost).
enum : int { kMapContiguous = 0, kMapStrided = 1 };

// Every apply maps (unit, lane) to at most one row and returns, on the lane
// that owns the row, w = z_s x_row - (H x)_row.  The vector type VV sets the
// arithmetic precision (float2: FP32, double2: FP64 with FP32 values promoted).

__device__ __forceinline__ void cfma_r(double2& acc, float v, double2 x) { cfma_r(acc, (double)v, x); }

// four consecutive complex entries starting at a 32-byte (float2) or 64-byte
// (double2) aligned address
__device__ __forceinline__ void load4(const float2* p, float2 (&x)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 2);
    x[0] = make_float2(a.x, a.y); x[1] = make_float2(a.z, a.w);
    x[2] = make_float2(b.x, b.y); x[3] = make_float2(b.z, b.w);
}
__device__ __forceinline__ void load4(const double2* p, double2 (&x)[4]) {
    x[0] = p[0]; x[1] = p[1]; x[2] = p[2]; x[3] = p[3];
}
__device__ __forceinline__ void load4(const float4* p, float4 (&x)[4]) {
    x[0] = p[0]; x[1] = p[1]; x[2] = p[2]; x[3] = p[3];
}

// acc += the accumulator of the lane at distance o (xor), for the row sums
// split over several lanes
__device__ __forceinline__ void lane_add(double2& acc, int o) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
}
__device__ __forceinline__ void lane_add(float2& acc, int o) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
}
__device__ __forceinline__ void lane_add(float4& acc, int o) {   // compensated: DF sums
    float4 w;
    w.x = __shfl_xor_sync(0xffffffffu, acc.x, o);
    w.y = __shfl_xor_sync(0xffffffffu, acc.y, o);
    w.z = __shfl_xor_sync(0xffffffffu, acc.z, o);
    w.w = __shfl_xor_sync(0xffffffffu, acc.w, o);
    acc = vadd_acc(acc, w);
}

template <typename R, int LPR>
struct ApplyCSR {
    static constexpr int kRowsPerUnit = 32 / LPR;
    static constexpr int kMap = kMapContiguous;
    const int* rowptr;
    const int* col;
    const R* val;
    int64_t n;
    int64_t nnz;
    unsigned long long* dbg;

    template <typename VV>
    __device__ __forceinline__ bool operator()(int64_t unit, int lane, VV zs, const VV* x,
                                               int64_t& row, VV& w) const {
        const int sub = lane / LPR, l = lane % LPR;
        row = unit * kRowsPerUnit + sub;
        VV acc = vzero<VV>();
        if (row < n) {
            const int e0 = rowptr[row], e1 = rowptr[row + 1];
            if (chk(dbg, 1, e0, nnz + 1) && chk(dbg, 2, e1, nnz + 1))
                for (int e = e0 + l; e < e1; e += LPR) {
                    const int c = ld_stream(col + e);
                    if (chk(dbg, 3, c, n)) cfma_r(acc, ld_stream(val + e), x[c]);
                }
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) lane_add(acc, o);
        if (row < n && l == 0) {
            w = vsub(vcfma(zs, x[row], vzero<VV>()), acc);
            return true;
        }
        return false;
    }
    // the row whose term (unit, lane) adds to the apply's r^T q partial
    __device__ __forceinline__ bool row_of(int64_t unit, int lane, int64_t& row) const {
        row = unit * kRowsPerUnit + lane / LPR;
        return row < n && lane % LPR == 0;
    }
};

// 4x4-blocked sliced ELL: a unit is 8 block rows (32 rows); slot s of unit u
// holds, for each of its 8 block rows, one column-block index (or -1 for
// padding) and one dense 4x4 block stored row-major.  Lane = 4 * block row +
// row within the block, so a warp's load of one slot is contiguous.
template <typename R>
struct ApplyBSR4 {
    static constexpr int kRowsPerUnit = 32;
    static constexpr int kMap = kMapContiguous;
    const int* unit_off;     // [nunits + 1] first slot of each unit
    const int* bcol;         // [slots][8]
    const R* bval;           // [slots][8][4][4]
    int64_t n;
    int64_t nslots;
    unsigned long long* dbg;

    __device__ __forceinline__ static void load_row(const float* p, float (&v)[4]) {
        const float4 t = ld_stream(reinterpret_cast<const float4*>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ __forceinline__ static void load_row(const double* p, double (&v)[4]) {
        const double2 a = ld_stream(reinterpret_cast<const double2*>(p));
        const double2 b = ld_stream(reinterpret_cast<const double2*>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }

    template <typename VV>
    __device__ __forceinline__ void block_fma(VV& acc, int cb, const R (&v)[4], const VV* x) const {
        if (cb >= 0 && chk(dbg, 5, (long long)cb * 4 + 3, n)) {
            VV xv[4];
            load4(x + (size_t)cb * 4, xv);
#pragma unroll
            for (int j = 0; j < 4; ++j) cfma_r(acc, v[j], xv[j]);
        }
    }

    template <typename VV>
    __device__ __forceinline__ bool operator()(int64_t unit, int lane, VV zs, const VV* x,
                                               int64_t& row, VV& w) const {
        const int br = lane >> 2, rr = lane & 3;
        row = unit * 32 + lane;
        int s0 = unit_off[unit], s1 = unit_off[unit + 1];
        if (!chk(dbg, 4, s1, nslots + 1) || !chk(dbg, 4, s0, s1 + 1)) s0 = s1 = 0;
        VV acc = vzero<VV>();
        constexpr int kG = SCOCG_BSR4_GROUP;
        for (int s = s0; s < s1; s += kG) {           // kG slots in flight; the last group predicated
            int cb[kG];
            R v[kG][4];
#pragma unroll
            for (int j = 0; j < kG; ++j) {
                if (s + j < s1) {
                    cb[j] = ld_stream(bcol + (size_t)(s + j) * 8 + br);
                    load_row(bval + ((size_t)(s + j) * 8 + br) * 16 + rr * 4, v[j]);
                } else {
                    cb[j] = -1;
                }
            }
#pragma unroll
            for (int j = 0; j < kG; ++j) block_fma(acc, cb[j], v[j], x);
        }
        if (row < n) {
            w = vsub(vcfma(zs, x[row], vzero<VV>()), acc);
            return true;
        }
        return false;
    }
    // the row whose term (unit, lane) adds to the apply's r^T q partial
    __device__ __forceinline__ bool row_of(int64_t unit, int lane, int64_t& row) const {
        row = unit * 32 + lane;
        return row < n;
    }
};

// Exchange of complex accumulators between lanes.
__device__ __forceinline__ float2 shfl_xor_v(float2 v, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ double2 shfl_xor_v(double2 v, int o) {
    return make_double2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// The same 4x4-blocked sliced ELL with each 4x4 block stored column-major,
// applied by column lanes (complex64 vectors): lane = 4 * block row + cc takes
// column cc of each block and the single entry x[4 cb + cc], and accumulates
// its contribution to all four rows of the block row.  The unit's column-block
// indices are read first, then four slots of H and x at a time; a
// reduce-scatter over the block row's four lanes leaves row 4 * block row + cc
// in lane 4 * block row + cc.  Each x entry is read by one lane per slot
// (instead of four), which shortens the gather; with compensated vectors the
// four accumulators cost more than the gather saves, so those keep the row
// lanes above.
template <typename R>
struct ApplyBSR4C {
    static constexpr int kRowsPerUnit = 32;
    static constexpr int kMap = kMapContiguous;
    static constexpr int kMaxSlots = 8;      // longer units take the loop below in chunks of 8
    const int* unit_off;
    const int* bcol;
    const float* bvalc;      // [slots][8][4 columns][4 rows]
    int64_t n;
    int64_t nslots;
    unsigned long long* dbg;

    template <typename VV>   // float2, or double2 for the FP64 residual replacement
    __device__ __forceinline__ bool operator()(int64_t unit, int lane, VV zs, const VV* x,
                                               int64_t& row, VV& w) const {
        const int br = lane >> 2, cc = lane & 3;
        row = unit * 32 + lane;
        int s0 = unit_off[unit], s1 = unit_off[unit + 1];
        if (!chk(dbg, 4, s1, nslots + 1) || !chk(dbg, 4, s0, s1 + 1)) s0 = s1 = 0;
        VV acc[4] = {vzero<VV>(), vzero<VV>(), vzero<VV>(), vzero<VV>()};
        for (int c0 = s0; c0 < s1; c0 += kMaxSlots) {
            const int ns = min(s1 - c0, kMaxSlots);
            int cb[kMaxSlots];
#pragma unroll
            for (int j = 0; j < kMaxSlots; ++j) cb[j] = j < ns ? ld_stream(bcol + (size_t)(c0 + j) * 8 + br) : -1;
#pragma unroll
            for (int j0 = 0; j0 < kMaxSlots; j0 += 4) {
                if (j0 >= ns) break;
                float4 v[4];
                VV xv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    v[j] = j0 + j < ns ? ld_stream(reinterpret_cast<const float4*>(bvalc + ((size_t)(c0 + j0 + j) * 8 + br) * 16 + cc * 4))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                    const int c = cb[j0 + j];
                    xv[j] = (c >= 0 && chk(dbg, 5, (long long)c * 4 + 3, n)) ? x[(size_t)c * 4 + cc] : vzero<VV>();
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    cfma_r(acc[0], v[j].x, xv[j]); cfma_r(acc[1], v[j].y, xv[j]);
                    cfma_r(acc[2], v[j].z, xv[j]); cfma_r(acc[3], v[j].w, xv[j]);
                }
            }
        }
        // reduce-scatter over the four lanes of the block row (xor 2, then xor 1)
        const bool b1 = (cc >> 1) & 1, b0 = cc & 1;
        VV k0 = b1 ? acc[2] : acc[0], k1 = b1 ? acc[3] : acc[1];
        const VV t0 = shfl_xor_v(b1 ? acc[0] : acc[2], 2), t1 = shfl_xor_v(b1 ? acc[1] : acc[3], 2);
        k0.x += t0.x; k0.y += t0.y; k1.x += t1.x; k1.y += t1.y;
        const VV t = shfl_xor_v(b0 ? k0 : k1, 1);
        VV mine = b0 ? k1 : k0;
        mine.x += t.x; mine.y += t.y;
        if (row < n) {
            w = vsub(vcfma(zs, x[row], vzero<VV>()), mine);
            return true;
        }
        return false;
    }
    // the row whose term (unit, lane) adds to the apply's r^T q partial
    __device__ __forceinline__ bool row_of(int64_t unit, int lane, int64_t& row) const {
        row = unit * 32 + lane;
        return row < n;
    }
};

// The blocked apply of each vector precision: column lanes for complex64,
// row lanes otherwise.
template <typename R> struct BsrApply { using T = ApplyBSR4<typename ValT<R>::T>; };
template <> struct BsrApply<float> { using T = ApplyBSR4C<float>; };

// ---------------------------------------------------------------- arguments
template <typename R>
struct SolveArgs {
    using V = typename Vec<R>::T;
    int64_t n;
    int64_t nunits;
    int rows_per_unit;
    V* r;
    V* q;
    const double2* b;          // rhs, complex128 [n]
    const V* cvec;             // dense projections [nproj][n] in vector precision, or null
    const int64_t* cidx;       // unit projections [nproj], or null
    int nproj;
    // MIXED: seed direction and compensated seed solution; FP64 apply for replacement
    V* p_seed;
    V* x_hi;
    V* x_lo;
    double2* xd;               // FP64 copy of x used by the replacement apply
    int replace_every;
    // shifts
    int K;
    const double2* z;
    int seed;
    int allow_switch;
    double tol;
    int max_iter;
    ShiftState S;
    // per-CTA partials
    double* partA;             // value-major [4][grid]
    double* partB;             // value-major [strideB][grid]
    double* partC;             // [grid][kPartC]
    int strideB;
    GridSync sync;
    SolveStats* stats;
    double2* G;                // out [nproj][K] for this right-hand side
    int debug_inject;
    unsigned long long* dbg;   // checked builds: first out-of-range index
    int* trace;                // checked builds: host-mapped (iteration, phase) per CTA
    unsigned long long* phase_ns;  // phase-timer builds: [grid][8] accumulated ns
    // full-vector mode (FP64 only): per-shift solutions and directions, [K][n];
    // needs K * kFullSmem bytes of dynamic shared memory
    double2* Xf;
    double2* Pf;
    // continuation: the state a solve stopped at max_iter leaves (written at
    // exit when non-null), and resume = 1 to start from it instead of r_0 = b
    ResumeState* rstate;
    int resume;
};
constexpr int kFullSmem = 3 * 16 + 4;   // per shift: 1/pi_n, beta^k, alpha^k, active flag

// Shared per-CTA copy of the seed scalars; every CTA holds identical values.
// CTA scratch of the block sums: per warp 3 + 2 kMaxProj values, or (FP64
// block sums) kScratchNV values per thread
constexpr int kScratchNV = 5;
constexpr int kScratch = kWarps * (3 + 2 * kMaxProj) > kScratchNV * kBlock ? kWarps * (3 + 2 * kMaxProj)
                                                                          : kScratchNV * kBlock;
struct SeedScalars {
    double2 alpha, alpha_prev, beta_prev, rho, rho_prev, zs;
    double2 t2;                 // alpha_n beta_{n-1} / alpha_{n-1}
    double rnorm, bnorm, rn_b;  // rn_b = ||r_{n+1}|| / ||b||
    double2 beta_next;          // rho_{n+1} / rho_n, before it becomes beta_prev
    double rnorm_next;          // ||r_{n+1}||, before it becomes rnorm
    int seed, active, n;
    int replace_on, n_switch, n_replace;
    long long shift_iters;
    double2 cr_cur[kMaxProj];   // c_m^T r_n
    double2 cr_next[kMaxProj];  // c_m^T r_{n+1}
    double red[4 + 2 * kMaxProj + 4];
    double scratch[kScratch];
};

// residual estimate of a shift from the seed residual norm and its pi
__device__ __forceinline__ double shift_resid(double rnorm, double2 pi, double bnorm) {
    return rnorm / (cabs_(pi) * bnorm);
}

// Fixed-order complex dot contribution c^T r in FP64
__device__ __forceinline__ void acc_dot(double2& s, double2 a, double2 b) {
    s.x = fma(a.x, b.x, fma(-a.y, b.y, s.x));
    s.y = fma(a.x, b.y, fma(a.y, b.x, s.y));
}

}  // namespace scocg
