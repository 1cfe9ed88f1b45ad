// The Lanczos-based parts of the library, all in FP64 on real vectors:
//
// * scocg_ground_state: the ground state of a real symmetric H by the Lanczos
//   method followed by the conjugate-gradient method used as inverse
//   iteration, the two repeated until the residual norm is small enough
//   (Sec. II.B).  The vector it returns is the starting point of the
//   excitation spectra: c|psi_0> and c+|psi_0> (scocg_excite, hubbard.cu) are
//   right-hand sides of the shifted solve.
// * scocg_krylov_sd: Green's functions by subspace diagonalisation in the
//   Krylov subspace K_nu(H, b) (Sec. III.B, Eq. Ham_in_KS): the eigenpairs of
//   the Lanczos tridiagonal T and the projections c_m^T v_j give
//   G_m(z) = sum_a (c_m^T w_a)(w_a^T b) / (z - e_a).
//
// One ground-state cycle:
//   Lanczos, m steps from psi (no reorthogonalization):
//     w = H v_j - beta_{j-1} v_{j-1};  alpha_j = v_j^T w;  w -= alpha_j v_j;
//     beta_j = ||w||;  v_{j+1} = w / beta_j  (stop when beta_j vanishes)
//   lowest eigenpair (theta, s) of T = tridiag(beta, alpha, beta): Sturm
//     multisection, then inverse iteration with a pivoted tridiagonal LU
//   psi = V s / ||V s||;  E = psi^T H psi;  res = ||H psi - E psi||
//   stop if res <= tol; else CG on (H - sigma) y = psi, sigma = E - res
//     (below the lowest eigenvalue once psi is close to it, so H - sigma is
//     positive definite), y = 0 first, at most cg_steps steps, stopped at a
//     relative residual of 1e-10 or when p^T (H - sigma) p <= 0; psi = y / ||y||.
//
// GPU layout: the Lanczos basis V[m][N] (FP64) stays in HBM during the cycle,
// so the Ritz vector is one pass over it instead of a second Lanczos run; all
// scalars stay on the device.  Each reduction is written as per-block partials
// that every consuming block adds in the same order, and every flag a kernel
// decides is stored per step, so no launch reads a value that it also writes
// and the host synchronises once per cycle to read E and res.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "api_internal.h"
#include "common.cuh"
#include "vector_ops.cuh"

namespace scocg {
namespace {

constexpr double kCgRtol = 1e-10;
constexpr int kMaxLanczos = 1024;

// y = (H - sigma) x - beta x_prev on the int32 CSR with FP64 values, 8 lanes
// per row (the 4 row groups of a warp take consecutive rows, so every lane of
// a warp runs the same number of outer steps); partial of x^T y per block.
__global__ void __launch_bounds__(kVecBlock) k_csr_hx(int64_t n, const int* rowptr, const int* col,
                                                      const double* val, const double* x, double* y,
                                                      const double* xprev, const double* beta, double sigma,
                                                      const int* skip, double* part) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31, sub = lane & 7;
    const int64_t gw = ((blockIdx.x * (int64_t)kVecBlock + threadIdx.x) >> 5) * 4;   // first row group of the warp
    const int64_t ng = ((int64_t)gridDim.x * kVecBlock) >> 3;
    const double bp = (xprev && beta) ? *beta : 0.0;
    double acc = 0.0;
    for (int64_t base = gw; base < n; base += ng) {
        const int64_t i = base + (lane >> 3);
        double s = 0.0;
        if (i < n)
            for (int k = rowptr[i] + sub; k < rowptr[i + 1]; k += 8) s = fma(val[k], x[col[k]], s);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        if (i < n && sub == 0) {
            const double xi = x[i];
            double yi = fma(-sigma, xi, s);
            if (xprev) yi = fma(-bp, xprev[i], yi);
            y[i] = yi;
            acc = fma(xi, yi, acc);
        }
    }
    block_partial(acc, part);
}

__device__ __forceinline__ bool lead() { return blockIdx.x == 0 && threadIdx.x == 0; }

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)kVecBlock + threadIdx.x; i < (n); i += (int64_t)gridDim.x * kVecBlock)

// (H x) for the rows of one unit of the 4x4-blocked sliced ELL (FP64 blocks):
// a warp takes a unit of 8 block rows (lane = 4 * block row + row within it);
// each slot is one contiguous 1 KB line of blocks, of which a lane reads the
// four values of its row, and the four entries of x of the block's column;
// four slots are in flight at a time.
__device__ __forceinline__ double bsr4_row(int64_t u, int lane, const int* unit_off, const int* bcol,
                                           const double* bval, const double* x) {
    const int br = lane >> 2, rr = lane & 3;
    const int s0 = unit_off[u], s1 = unit_off[u + 1];
    double hs = 0.0;
    for (int s = s0; s < s1; s += 4) {
        int cb[4];
        double2 va[4], vb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            cb[q] = s + q < s1 ? __ldcs(bcol + (size_t)(s + q) * 8 + br) : -1;
            if (cb[q] >= 0) {
                const double2* v = reinterpret_cast<const double2*>(bval + ((size_t)(s + q) * 8 + br) * 16 + rr * 4);
                va[q] = __ldcs(v);
                vb[q] = __ldcs(v + 1);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (cb[q] < 0) continue;
            const double2* xp = reinterpret_cast<const double2*>(x + (size_t)cb[q] * 4);
            const double2 xa = xp[0], xb = xp[1];
            hs = fma(va[q].x, xa.x, hs);
            hs = fma(va[q].y, xa.y, hs);
            hs = fma(vb[q].x, xb.x, hs);
            hs = fma(vb[q].y, xb.y, hs);
        }
    }
    return hs;
}

// The operator of k_csr_hx on the 4x4-blocked layout.
__global__ void __launch_bounds__(kVecBlock) k_bsr4_hx(int64_t nunits, const int* unit_off, const int* bcol,
                                                       const double* bval, int64_t n, const double* x, double* y,
                                                       const double* xprev, const double* beta, double sigma,
                                                       const int* skip, double* part) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)kVecBlock + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * kVecBlock) >> 5;
    const double bp = (xprev && beta) ? *beta : 0.0;
    double acc = 0.0;
    for (int64_t u = w0; u < nunits; u += nw) {
        const double hs = bsr4_row(u, lane, unit_off, bcol, bval, x);
        const int64_t row = u * 32 + lane;
        if (row < n) {
            const double xi = x[row];
            double yi = fma(-sigma, xi, hs);
            if (xprev) yi = fma(-bp, xprev[row], yi);
            y[row] = yi;
            acc = fma(xi, yi, acc);
        }
    }
    block_partial(acc, part);
}

// KR-SD's Lanczos recursion in one cooperative launch (4x4-blocked layout,
// unit projections), two grid barriers per step.  With w_{-1} = b and
// beta_{-1} = ||b||, step j forms v_j = w_{j-1} / beta_{j-1} on the fly:
//   phase 1: w_j = (H w_{j-1}) / beta_{j-1} - beta_{j-1} v_{j-1} and
//            v_j for the own rows, partial of v_j^T w_j; CTA 0 records
//            c_m^T v_j = w_{j-1}[idx_m] / beta_{j-1}
//   barrier; alpha_j = sum of the partials (same order in every CTA)
//   phase 2: w_j -= alpha_j v_j, partial of ||w_j||^2
//   barrier; beta_j = sqrt(sum); the recursion ends after step j when
//            j + 1 = nu or beta_j <= 1e-12 max_i(|alpha_i| + beta_i + beta_{i-1})
// A row is always handled by the warp of its unit; v and w alternate between
// two buffers each, so a buffer is rewritten only after the barrier that ends
// every gather of its old contents.  Waits are bounded (GridSync timeout).
struct KrylovArgs {
    int64_t n, nunits;
    const int* unit_off;
    const int* bcol;
    const double* bval;
    const double* b;
    double* V[2];
    double* W[2];
    int nu, M;
    const int64_t* idx;
    double* P;
    double* alpha;
    double* beta;
    int* kdim;
    double* part_a;   // partials of v_j^T w_j
    double* part_b;   // partials of ||b||^2, then of ||w_j||^2
    GridSync sync;
};

__global__ void __launch_bounds__(kVecBlock) k_krylov_lanczos(KrylovArgs a) {
    const int lane = threadIdx.x & 31;
    const int G = gridDim.x;
    const int64_t w0 = (blockIdx.x * (int64_t)kVecBlock + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)G * kVecBlock) >> 5;
    unsigned long long epoch = 0;
    // step scalars: roots and divisions by thread 0 only, broadcast through
    // shared memory (done by every thread they would load the FP64 pipe with
    // as many instructions as the operator itself)
    __shared__ double s_bprev, s_inv;
    __shared__ int s_end;
    double tn = 0.0;   // thread 0's running max of |alpha_i| + beta_i + beta_{i-1}
    // ||b||
    double acc = 0.0;
    GRID_STRIDE(i, a.n) acc = fma(a.b[i], a.b[i], acc);
    block_partial(acc, a.part_b);
    if (!grid_barrier(a.sync, epoch)) return;
    {
        const double s0 = sum_partials(a.part_b, G);
        if (threadIdx.x == 0) { s_bprev = sqrt(s0); s_inv = 1.0 / s_bprev; }
        __syncthreads();
    }
    const double* wprev = a.b;
    for (int j = 0; j < a.nu; ++j) {
        double* vcur = a.V[j & 1];
        const double* vprev = a.V[(j + 1) & 1];
        double* wcur = a.W[j & 1];
        const double bprev = s_bprev;   // beta_{j-1}
        const double inv = s_inv;
        if (blockIdx.x == 0 && threadIdx.x < a.M) a.P[(size_t)threadIdx.x * a.nu + j] = wprev[a.idx[threadIdx.x]] * inv;
        acc = 0.0;
        for (int64_t u = w0; u < a.nunits; u += nw) {
            const double hs = bsr4_row(u, lane, a.unit_off, a.bcol, a.bval, wprev);
            const int64_t row = u * 32 + lane;
            if (row < a.n) {
                const double vi = wprev[row] * inv;
                double wi = hs * inv;
                if (j > 0) wi = fma(-bprev, vprev[row], wi);
                vcur[row] = vi;
                wcur[row] = wi;
                acc = fma(vi, wi, acc);
            }
        }
        block_partial(acc, a.part_a);
        if (!grid_barrier(a.sync, epoch)) return;
        const double al = sum_partials(a.part_a, G);
        acc = 0.0;
        for (int64_t u = w0; u < a.nunits; u += nw) {
            const int64_t row = u * 32 + lane;
            if (row < a.n) {
                const double wi = fma(-al, vcur[row], wcur[row]);
                wcur[row] = wi;
                acc = fma(wi, wi, acc);
            }
        }
        // part_b is read after the next barrier and rewritten only after the
        // first barrier of the next step, by which time every CTA has read it
        block_partial(acc, a.part_b);
        if (!grid_barrier(a.sync, epoch)) return;
        const double bsq = sum_partials(a.part_b, G);
        if (threadIdx.x == 0) {
            const double be = sqrt(bsq);
            tn = fmax(tn, fabs(al) + be + (j > 0 ? bprev : 0.0));
            const bool end = (j + 1 == a.nu) || !(be > 1e-12 * tn);
            if (blockIdx.x == 0) {
                a.alpha[j] = al;
                a.beta[j] = be;
                if (end) *a.kdim = j + 1;
            }
            s_end = end;
            s_bprev = be;
            s_inv = 1.0 / be;
        }
        __syncthreads();
        if (s_end) break;
        wprev = wcur;
    }
}


// KR-SD's recursion for several right-hand sides at once (one per slot,
// s < T): the vectors are [n][T] with the slot fastest, so that every read of
// H's 4x4 blocks serves all T recursions, and each slot has its own scalars,
// projections and end.  Lane = T * (block row within the warp step) + slot.
// Per step the same operations as k_krylov_lanczos, slot by slot; a slot that
// has ended (or holds no right-hand side) keeps running with zero vectors and
// records nothing.  Waits are bounded (GridSync timeout).
struct KrylovBlockArgs {
    int64_t n, nunits;
    const int* unit_off;
    const int* bcol;
    const double* bval;
    const double* B;          // [n][T] the right-hand sides
    double* V[2];
    double* W[2];             // [n][T]
    int nu, M, nslot;         // steps, unit projections per slot, slots in use
    const int64_t* idx;       // [T][M]
    double* P;                // [T][M][nu] c_m^T v_j
    double* alpha;            // [T][nu]
    double* beta;             // [T][nu]
    double* bnorm;            // [T]
    int* kdim;                // [T]
    double* part_a;           // [T][G] partials of v_j^T w_j
    double* part_b;           // [T][G] partials of ||b||^2, then of ||w_j||^2
    GridSync sync;
};

// the CTA's partial of each slot's per-thread values into part[slot * G + cta]
template <int T>
__device__ __forceinline__ void slot_partial(double v, double (*s_w)[T], double* part, int G) {
#pragma unroll
    for (int o = T; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);   // the warp's lanes of one slot
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < T) s_w[warp][lane] = v;
    __syncthreads();
    if (threadIdx.x < T) {
        double t = 0.0;
        for (int w = 0; w < kVecBlock / 32; ++w) t += s_w[w][threadIdx.x];
        part[(size_t)threadIdx.x * G + blockIdx.x] = t;
    }
    __syncthreads();
}

// every CTA sums each slot's partials over the CTAs in the same order
template <int T>
__device__ __forceinline__ void slot_sums(const double* part, int G, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = warp; t < T; t += kVecBlock / 32) {
        double acc = 0.0;
        for (int c = lane; c < G; c += 32) acc += __ldcg(part + (size_t)t * G + c);
        acc = warp_sum(acc);
        if (lane == 0) out[t] = acc;
    }
    __syncthreads();
}

template <int T>
__global__ void __launch_bounds__(kVecBlock) k_krylov_block(KrylovBlockArgs a) {
    constexpr int RPW = 32 / T;              // block rows per warp step
    constexpr int kW = kVecBlock / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / T, cl = lane % T;
    const int G = gridDim.x, cta = blockIdx.x;
    __shared__ double s_w[kW][T];
    __shared__ double s_al[T], s_b2[T], s_bprev[T], s_inv[T], s_tn[T];
    __shared__ int s_end[T];
    unsigned long long epoch = 0;
    const int64_t nbr = a.n / 4;
    const int64_t bfirst = (int64_t)cta * nbr / G + warp * RPW + sub, bend = (int64_t)(cta + 1) * nbr / G;
    constexpr int64_t bstep = (int64_t)kW * RPW;
    const double* wprev = a.B;
    // ||b_s||
    double acc = 0.0;
    for (int64_t B = bfirst; B < bend; B += bstep)
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const double x = wprev[((size_t)B * 4 + rr) * T + cl];
            acc = fma(x, x, acc);
        }
    slot_partial<T>(acc, s_w, a.part_b, G);
    if (!grid_barrier(a.sync, epoch)) return;
    slot_sums<T>(a.part_b, G, s_b2);
    if (threadIdx.x < T) {
        const int t = threadIdx.x;
        const double bn = sqrt(s_b2[t]);
        s_end[t] = t >= a.nslot || !(bn > 0.0);
        s_bprev[t] = bn;
        s_inv[t] = s_end[t] ? 0.0 : 1.0 / bn;
        s_tn[t] = 0.0;
        if (cta == 0) {
            a.bnorm[t] = bn;
            a.kdim[t] = 0;
        }
    }
    __syncthreads();
    for (int j = 0; j < a.nu; ++j) {
        double* vcur = a.V[j & 1];
        const double* vprev = a.V[(j + 1) & 1];
        double* wcur = a.W[j & 1];
        if (cta == 0)
            for (int p = threadIdx.x; p < T * a.M; p += kVecBlock) {
                const int t = p / a.M;
                if (!s_end[t]) a.P[(size_t)p * a.nu + j] = wprev[(size_t)a.idx[p] * T + t] * s_inv[t];
            }
        const double inv = s_inv[cl], bprev = s_bprev[cl];
        acc = 0.0;
        for (int64_t B = bfirst; B < bend; B += bstep) {
            double hs[4] = {0.0, 0.0, 0.0, 0.0};
            const int64_t u = B >> 3;
            const int br = (int)(B & 7);
            const int s0 = a.unit_off[u], s1 = a.unit_off[u + 1];
            for (int sl = s0; sl < s1; ++sl) {
                const int cb = ld_stream(a.bcol + (size_t)sl * 8 + br);
                if (cb < 0) continue;
                double xv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) xv[q] = wprev[((size_t)cb * 4 + q) * T + cl];
                // the block's 16 values (row-major) as eight 16-byte loads
                const double2* hb = reinterpret_cast<const double2*>(a.bval + ((size_t)sl * 8 + br) * 16);
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    const double2 h01 = ld_stream(hb + 2 * rr), h23 = ld_stream(hb + 2 * rr + 1);
                    hs[rr] = fma(h01.x, xv[0], hs[rr]);
                    hs[rr] = fma(h01.y, xv[1], hs[rr]);
                    hs[rr] = fma(h23.x, xv[2], hs[rr]);
                    hs[rr] = fma(h23.y, xv[3], hs[rr]);
                }
            }
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const size_t o = ((size_t)B * 4 + rr) * T + cl;
                const double vi = wprev[o] * inv;
                double wi = hs[rr] * inv;
                if (j > 0) wi = fma(-bprev, vprev[o], wi);
                vcur[o] = vi;
                wcur[o] = wi;
                acc = fma(vi, wi, acc);
            }
        }
        slot_partial<T>(acc, s_w, a.part_a, G);
        if (!grid_barrier(a.sync, epoch)) return;
        slot_sums<T>(a.part_a, G, s_al);
        const double al = s_al[cl];
        acc = 0.0;
        for (int64_t B = bfirst; B < bend; B += bstep)
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const size_t o = ((size_t)B * 4 + rr) * T + cl;
                const double wi = fma(-al, vcur[o], wcur[o]);
                wcur[o] = wi;
                acc = fma(wi, wi, acc);
            }
        slot_partial<T>(acc, s_w, a.part_b, G);
        if (!grid_barrier(a.sync, epoch)) return;
        slot_sums<T>(a.part_b, G, s_b2);
        if (threadIdx.x < T) {
            const int t = threadIdx.x;
            const double be = sqrt(s_b2[t]);
            bool end = s_end[t] != 0;
            if (!end) {
                s_tn[t] = fmax(s_tn[t], fabs(s_al[t]) + be + (j > 0 ? s_bprev[t] : 0.0));
                end = (j + 1 == a.nu) || !(be > 1e-12 * s_tn[t]);
                if (cta == 0) {
                    a.alpha[(size_t)t * a.nu + j] = s_al[t];
                    a.beta[(size_t)t * a.nu + j] = be;
                    if (end) a.kdim[t] = j + 1;
                }
            }
            s_end[t] = end;
            s_bprev[t] = be;
            s_inv[t] = end ? 0.0 : 1.0 / be;
        }
        __syncthreads();
        bool live = false;
#pragma unroll
        for (int t = 0; t < T; ++t) live = live || !s_end[t];
        if (!live) break;
        wprev = wcur;
    }
}

// The same recursions with compensated FP32 arithmetic (SCOCG_MIXED_DF
// handles): H's FP32 4x4 blocks, vector entries as float pairs hi + lo, the
// products exact to the pair precision and the sums by TwoSum, so that the
// recursion runs on the FP32 pipe (the FP64 one bounds the version above);
// the step scalars stay FP64.  Two rows of a block row share each paired
// FP32 instruction of the apply.
__device__ __forceinline__ void pk_acc_fx(float2& ah, float2& al, float2 v, float xh, float xl) {
    const float2 xh2 = make_float2(xh, xh);
    const float2 p = pk_mul(v, xh2);
    float2 e = pk_fma(v, xh2, pk_neg(p));
    e = pk_fma(v, make_float2(xl, xl), e);
    float2 s, t;
    pk_two_sum(ah, p, s, t);
    ah = s;
    al = pk_add(al, pk_add(t, e));
}
__device__ __forceinline__ dfs df_of(double v) {
    const float hi = (float)v;
    return dfs{hi, (float)(v - (double)hi)};
}
__device__ __forceinline__ dfs df_ld(const float2* p) {
    const float2 v = *p;
    return dfs{v.x, v.y};
}

struct KrylovBlockDfArgs {
    int64_t n, nunits;
    const int* unit_off;
    const int* bcol;
    const float* bval;        // FP32 4x4 blocks, row-major
    const float2* B;          // [n][T] (hi, lo)
    float2* V[2];
    float2* W[2];
    int nu, M, nslot;
    const int64_t* idx;
    double* P;
    double* alpha;
    double* beta;
    double* bnorm;
    int* kdim;
    double* part_a;
    double* part_b;
    GridSync sync;
};

template <int T>
__global__ void __launch_bounds__(kVecBlock) k_krylov_block_df(KrylovBlockDfArgs a) {
    constexpr int RPW = 32 / T;
    constexpr int kW = kVecBlock / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / T, cl = lane % T;
    const int G = gridDim.x, cta = blockIdx.x;
    __shared__ double s_w[kW][T];
    __shared__ double s_al[T], s_b2[T], s_bprev[T], s_inv[T], s_tn[T];
    __shared__ int s_end[T];
    unsigned long long epoch = 0;
    const int64_t nbr = a.n / 4;
    const int64_t bfirst = (int64_t)cta * nbr / G + warp * RPW + sub, bend = (int64_t)(cta + 1) * nbr / G;
    constexpr int64_t bstep = (int64_t)kW * RPW;
    const float2* wprev = a.B;
    dfs acc = {0.f, 0.f};
    for (int64_t B = bfirst; B < bend; B += bstep)
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const dfs x = df_ld(wprev + ((size_t)B * 4 + rr) * T + cl);
            df_acc_prod(acc, x, x);
        }
    slot_partial<T>(df_to(df_norm(acc.hi, acc.lo)), s_w, a.part_b, G);
    if (!grid_barrier(a.sync, epoch)) return;
    slot_sums<T>(a.part_b, G, s_b2);
    if (threadIdx.x < T) {
        const int t = threadIdx.x;
        const double bn = sqrt(s_b2[t]);
        s_end[t] = t >= a.nslot || !(bn > 0.0);
        s_bprev[t] = bn;
        s_inv[t] = s_end[t] ? 0.0 : 1.0 / bn;
        s_tn[t] = 0.0;
        if (cta == 0) {
            a.bnorm[t] = bn;
            a.kdim[t] = 0;
        }
    }
    __syncthreads();
    for (int j = 0; j < a.nu; ++j) {
        float2* vcur = a.V[j & 1];
        const float2* vprev = a.V[(j + 1) & 1];
        float2* wcur = a.W[j & 1];
        if (cta == 0)
            for (int p = threadIdx.x; p < T * a.M; p += kVecBlock) {
                const int t = p / a.M;
                if (!s_end[t]) a.P[(size_t)p * a.nu + j] = df_to(df_ld(wprev + (size_t)a.idx[p] * T + t)) * s_inv[t];
            }
        const dfs inv = df_of(s_inv[cl]), nbprev = df_of(-s_bprev[cl]);
        acc = dfs{0.f, 0.f};
        for (int64_t B = bfirst; B < bend; B += bstep) {
            float2 h01 = make_float2(0.f, 0.f), l01 = h01, h23 = h01, l23 = h01;   // rows (0, 1) and (2, 3)
            const int64_t u = B >> 3;
            const int br = (int)(B & 7);
            const int s0 = a.unit_off[u], s1 = a.unit_off[u + 1];
            for (int sl = s0; sl < s1; ++sl) {
                const int cb = ld_stream(a.bcol + (size_t)sl * 8 + br);
                if (cb < 0) continue;
                float2 xv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) xv[q] = wprev[((size_t)cb * 4 + q) * T + cl];
                const float4* hb = reinterpret_cast<const float4*>(a.bval + ((size_t)sl * 8 + br) * 16);
                const float4 r0 = ld_stream(hb), r1 = ld_stream(hb + 1), r2 = ld_stream(hb + 2), r3 = ld_stream(hb + 3);
                pk_acc_fx(h01, l01, make_float2(r0.x, r1.x), xv[0].x, xv[0].y);
                pk_acc_fx(h01, l01, make_float2(r0.y, r1.y), xv[1].x, xv[1].y);
                pk_acc_fx(h01, l01, make_float2(r0.z, r1.z), xv[2].x, xv[2].y);
                pk_acc_fx(h01, l01, make_float2(r0.w, r1.w), xv[3].x, xv[3].y);
                pk_acc_fx(h23, l23, make_float2(r2.x, r3.x), xv[0].x, xv[0].y);
                pk_acc_fx(h23, l23, make_float2(r2.y, r3.y), xv[1].x, xv[1].y);
                pk_acc_fx(h23, l23, make_float2(r2.z, r3.z), xv[2].x, xv[2].y);
                pk_acc_fx(h23, l23, make_float2(r2.w, r3.w), xv[3].x, xv[3].y);
            }
            pk_norm(h01, l01);
            pk_norm(h23, l23);
            const dfs hs[4] = {{h01.x, l01.x}, {h01.y, l01.y}, {h23.x, l23.x}, {h23.y, l23.y}};
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const size_t o = ((size_t)B * 4 + rr) * T + cl;
                const dfs vi = df_mul(df_ld(wprev + o), inv);
                dfs wi = df_mul(hs[rr], inv);
                if (j > 0) wi = df_add(wi, df_mul(nbprev, df_ld(vprev + o)));
                vcur[o] = make_float2(vi.hi, vi.lo);
                wcur[o] = make_float2(wi.hi, wi.lo);
                df_acc_prod(acc, vi, wi);
            }
        }
        slot_partial<T>(df_to(df_norm(acc.hi, acc.lo)), s_w, a.part_a, G);
        if (!grid_barrier(a.sync, epoch)) return;
        slot_sums<T>(a.part_a, G, s_al);
        const dfs nal = df_of(-s_al[cl]);
        acc = dfs{0.f, 0.f};
        for (int64_t B = bfirst; B < bend; B += bstep)
#pragma unroll
            for (int rr = 0; rr < 4; ++rr) {
                const size_t o = ((size_t)B * 4 + rr) * T + cl;
                const dfs wi = df_add(df_ld(wcur + o), df_mul(nal, df_ld(vcur + o)));
                wcur[o] = make_float2(wi.hi, wi.lo);
                df_acc_prod(acc, wi, wi);
            }
        slot_partial<T>(df_to(df_norm(acc.hi, acc.lo)), s_w, a.part_b, G);
        if (!grid_barrier(a.sync, epoch)) return;
        slot_sums<T>(a.part_b, G, s_b2);
        if (threadIdx.x < T) {
            const int t = threadIdx.x;
            const double be = sqrt(s_b2[t]);
            bool end = s_end[t] != 0;
            if (!end) {
                s_tn[t] = fmax(s_tn[t], fabs(s_al[t]) + be + (j > 0 ? s_bprev[t] : 0.0));
                end = (j + 1 == a.nu) || !(be > 1e-12 * s_tn[t]);
                if (cta == 0) {
                    a.alpha[(size_t)t * a.nu + j] = s_al[t];
                    a.beta[(size_t)t * a.nu + j] = be;
                    if (end) a.kdim[t] = j + 1;
                }
            }
            s_end[t] = end;
            s_bprev[t] = be;
            s_inv[t] = end ? 0.0 : 1.0 / be;
        }
        __syncthreads();
        bool live = false;
#pragma unroll
        for (int t = 0; t < T; ++t) live = live || !s_end[t];
        if (!live) break;
        wprev = wcur;
    }
}

// x [nslot][n] (FP64) -> y [n][T] as float pairs (hi, lo), zero past nslot
__global__ void k_to_slots_df(int64_t n, int T, int nslot, const double* x, float2* y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * T) return;
    const int64_t row = i / T;
    const int t = (int)(i % T);
    const double v = t < nslot ? x[(size_t)t * n + row] : 0.0;
    const float hi = (float)v;
    y[i] = make_float2(hi, (float)(v - (double)hi));
}

// x [nslot][n] -> y [n][T] (slot fastest), zero in the slots past nslot
__global__ void k_to_slots(int64_t n, int T, int nslot, const double* x, double* y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n * T) return;
    const int64_t row = i / T;
    const int t = (int)(i % T);
    y[i] = t < nslot ? x[(size_t)t * n + row] : 0.0;
}

// partial of x^T x
__global__ void __launch_bounds__(kVecBlock) k_norm_part(int64_t n, const double* x, double* part) {
    double acc = 0.0;
    GRID_STRIDE(i, n) { const double v = x[i]; acc = fma(v, v, acc); }
    block_partial(acc, part);
}

// dst = src / sqrt(sum of the partials); dst left as it is when that sum is
// zero or not finite (*ok = 0, written by the lead thread)
__global__ void __launch_bounds__(kVecBlock) k_scale_to(int64_t n, const double* src, double* dst,
                                                        const double* part, int G, int* ok) {
    __shared__ double s_inv;
    const double s = sum_partials(part, G);
    const bool good = s > 0.0 && isfinite(s);
    if (lead() && ok) *ok = good;
    if (!good) return;
    if (threadIdx.x == 0) s_inv = 1.0 / sqrt(s);   // one thread: roots and divisions are long FP64 chains
    __syncthreads();
    const double inv = s_inv;
    GRID_STRIDE(i, n) dst[i] = src[i] * inv;
}

// alpha_j = sum(part); w -= alpha_j v_j; partial of w^T w
__global__ void __launch_bounds__(kVecBlock) k_lz_ortho(int64_t n, int j, const double* v, double* w,
                                                        const double* part, int G, const int* stop, double* alpha,
                                                        double* part2) {
    if (stop[j]) return;
    const double a = sum_partials(part, G);
    if (lead()) alpha[j] = a;
    double acc = 0.0;
    GRID_STRIDE(i, n) {
        const double wi = fma(-a, v[i], w[i]);
        w[i] = wi;
        acc = fma(wi, wi, acc);
    }
    block_partial(acc, part2);
}

// beta_j = sqrt(sum(part2)); the recursion ends after step j when j + 1 = m or
// beta_j <= 1e-12 * max_i (|alpha_i| + beta_i + beta_{i-1}) (an invariant
// subspace, or a non-finite value); else v_{j+1} = w / beta_j.
__global__ void __launch_bounds__(kVecBlock) k_lz_next(int64_t n, int j, int m, const double* w, double* vnext,
                                                       const double* part2, int G, const double* alpha, double* beta,
                                                       double* tnorm, int* stop, int* kdim) {
    if (stop[j]) {
        if (lead()) stop[j + 1] = 1;
        return;
    }
    __shared__ double s_inv;
    __shared__ int s_end;
    const double bsq = sum_partials(part2, G);
    if (threadIdx.x == 0) {   // one thread: roots and divisions are long FP64 chains
        const double b = sqrt(bsq);
        const double tn = fmax(j ? tnorm[j - 1] : 0.0, fabs(alpha[j]) + b + (j ? beta[j - 1] : 0.0));
        const bool end = (j + 1 == m) || !(b > 1e-12 * tn);
        if (blockIdx.x == 0) {
            beta[j] = b;
            tnorm[j] = tn;
            stop[j + 1] = end;
            if (end) *kdim = j + 1;
        }
        s_end = end;
        s_inv = 1.0 / b;
    }
    __syncthreads();
    if (s_end) return;
    const double inv = s_inv;
    GRID_STRIDE(i, n) vnext[i] = w[i] * inv;
}

// Sturm count: the number of eigenvalues of the k x k tridiagonal T below x,
// = the number of sign changes in the leading principal minors
// P_i = det(T_i - x), P_0 = 1, P_{i+1} = (a_i - x) P_i - b_{i-1}^2 P_{i-1}
// (no division, so no FP64 divide per step).  A minor that vanishes (or
// falls below pivmin |P_i|) is replaced by -pivmin P_i, like a tiny negative
// pivot; both minors are rescaled by 2^-600 / 2^600 to stay in range.
// a and b2 (= b_{i-1}^2 at index i) are staged in shared memory by the caller.
__device__ int tri_count_below(const double* a, const double* b2, int k, double x, double pivmin) {
    int c = 0;
    double pm = 0.0, p = 1.0;   // P_{i-1}, P_i
    for (int i = 0; i < k; ++i) {
        double pn = fma(a[i] - x, p, -b2[i] * pm);
        if (fabs(pn) <= pivmin * fabs(p)) pn = -pivmin * p;
        if ((pn < 0.0) != (p < 0.0)) ++c;
        pm = p;
        p = pn;
        if (fabs(p) > 0x1p600) { p *= 0x1p-600; pm *= 0x1p-600; }
        else if (fabs(p) < 0x1p-600 && fabs(pm) < 0x1p-600) { p *= 0x1p600; pm *= 0x1p600; }
    }
    return c;
}

// stage alpha and the squared off-diagonals (b2[0] = 0) in shared memory
__device__ __forceinline__ void stage_tri(const double* alpha, const double* beta, int k, double* s_a, double* s_b2) {
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        s_a[i] = alpha[i];
        s_b2[i] = i > 0 ? beta[i - 1] * beta[i - 1] : 0.0;
    }
    __syncthreads();
}

// Lowest eigenpair of the k x k tridiagonal T (alpha on the diagonal, beta
// off it), one warp: multisection on the Sturm count (negative pivots of the
// LDL^T factorisation of T - x) inside the Gershgorin interval, 32 points per
// round, each lane counting at one point; then, in lane 0, three steps of
// inverse iteration with T - theta factorised by Gaussian elimination with
// partial pivoting (U with two superdiagonals).
__global__ void k_tri_lowest(const int* kdim, const double* alpha, const double* beta, double* s, double* work,
                             double* theta_out) {
    if (blockIdx.x != 0) return;
    __shared__ double s_a[kMaxLanczos], s_b2[kMaxLanczos];
    const int lane = threadIdx.x & 31;
    const int k = *kdim;
    const double* a = alpha;
    const double* b = beta;
    stage_tri(alpha, beta, k, s_a, s_b2);
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
        lo = fmin(lo, a[i] - r);
        hi = fmax(hi, a[i] + r);
    }
    const double scale = fmax(fmax(fabs(lo), fabs(hi)), 1e-300);
    const double eps = 2.220446049250313e-16;
    const double pivmin = eps * scale * 1e-3 + 1e-300;
    lo -= 2.0 * eps * scale + pivmin;
    hi += 2.0 * eps * scale + pivmin;
    auto count_below = [&](double x) { return tri_count_below(s_a, s_b2, k, x, pivmin); };
    // invariant: no eigenvalue below lo, at least one below hi (the same on every lane)
    for (int it = 0; it < 64 && hi - lo > 2.0 * eps * fmax(fabs(lo), fabs(hi)) + pivmin; ++it) {
        const double x = lo + (hi - lo) * ((double)(lane + 1) / 33.0);
        const unsigned above = __ballot_sync(0xffffffffu, count_below(x) >= 1);
        const int f = above ? __ffs(above) - 1 : 32;    // first point with an eigenvalue below it
        const double xf = __shfl_sync(0xffffffffu, x, f < 32 ? f : 31);
        const double xp = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
        if (f == 32) lo = xf;
        else { hi = xf; if (f > 0) lo = xp; }
    }
    if (lane != 0) return;
    const double th = 0.5 * (lo + hi);
    *theta_out = th;
    // LU of T - th with row interchanges: U0 diagonal, U1, U2 superdiagonals,
    // l multipliers, sw = 1 where rows i and i + 1 were exchanged
    double* U0 = work;
    double* U1 = work + k;
    double* U2 = work + 2 * k;
    double* l = work + 3 * k;
    double* sw = work + 4 * k;
    const double tiny = eps * scale + 1e-280;
    double r0 = a[0] - th, r1 = k > 1 ? b[0] : 0.0, r2 = 0.0;
    for (int i = 0; i + 1 < k; ++i) {
        const double c = b[i];                       // row i+1: (b_i, a_{i+1} - th, b_{i+1})
        const double d1 = a[i + 1] - th, d2 = i + 2 < k ? b[i + 1] : 0.0;
        if (fabs(r0) >= fabs(c)) {
            const double m = r0 != 0.0 ? c / r0 : 0.0;
            U0[i] = r0; U1[i] = r1; U2[i] = r2; l[i] = m; sw[i] = 0.0;
            r0 = d1 - m * r1; r1 = d2 - m * r2; r2 = 0.0;
        } else {
            const double m = r0 / c;
            U0[i] = c; U1[i] = d1; U2[i] = d2; l[i] = m; sw[i] = 1.0;
            const double n0 = r1 - m * d1, n1 = r2 - m * d2;
            r0 = n0; r1 = n1; r2 = 0.0;
        }
        if (fabs(U0[i]) < tiny) U0[i] = U0[i] < 0.0 ? -tiny : tiny;
    }
    U0[k - 1] = fabs(r0) < tiny ? (r0 < 0.0 ? -tiny : tiny) : r0;
    for (int i = 0; i < k; ++i) s[i] = 1.0 + (double)((i * 7919) % 13) / 13.0;
    for (int rep = 0; rep < 3; ++rep) {
        for (int i = 0; i + 1 < k; ++i) {
            if (sw[i] != 0.0) { const double t = s[i]; s[i] = s[i + 1]; s[i + 1] = t; }
            s[i + 1] -= l[i] * s[i];
        }
        for (int i = k - 1; i >= 0; --i) {
            double v = s[i];
            if (i + 1 < k) v -= U1[i] * s[i + 1];
            if (i + 2 < k) v -= U2[i] * s[i + 2];
            s[i] = v / U0[i];
        }
        double mx = 0.0;
        for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(s[i]));
        if (!(mx > 0.0) || !isfinite(mx)) break;
        double nr = 0.0;
        for (int i = 0; i < k; ++i) { s[i] /= mx; nr += s[i] * s[i]; }
        nr = sqrt(nr);
        for (int i = 0; i < k; ++i) s[i] /= nr;
    }
}

// psi = sum_{j < k} s_j v_j; partial of psi^T psi
__global__ void __launch_bounds__(kVecBlock) k_ritz(int64_t n, const int* kdim, const double* s, const double* V,
                                                    double* psi, double* part) {
    __shared__ double s_s[kMaxLanczos];
    const int k = *kdim;
    for (int j = threadIdx.x; j < k; j += kVecBlock) s_s[j] = s[j];
    __syncthreads();
    double acc = 0.0;
    GRID_STRIDE(i, n) {
        double v = 0.0;
        for (int j = 0; j < k; ++j) v = fma(s_s[j], V[(size_t)j * n + i], v);
        psi[i] = v;
        acc = fma(v, v, acc);
    }
    block_partial(acc, part);
}

// E = sum(part) (= psi^T H psi with h = H psi); partial of ||h - E psi||^2
__global__ void __launch_bounds__(kVecBlock) k_resid(int64_t n, const double* psi, const double* h,
                                                     const double* part, int G, double* part2, double* E_out) {
    const double E = sum_partials(part, G);
    if (lead()) *E_out = E;
    double acc = 0.0;
    GRID_STRIDE(i, n) {
        const double r = fma(-E, psi[i], h[i]);
        acc = fma(r, r, acc);
    }
    block_partial(acc, part2);
}

// *out = sqrt(sum(part)) (one block) or the plain sum
__global__ void __launch_bounds__(kVecBlock) k_sum_store(const double* part, int G, double* out, int take_sqrt) {
    const double s = sum_partials(part, G);
    if (threadIdx.x == 0) *out = take_sqrt ? sqrt(s) : s;
}

// y = 0; r = p = psi; partial of r^T r
__global__ void __launch_bounds__(kVecBlock) k_cg_init(int64_t n, const double* psi, double* y, double* r, double* p,
                                                       double* part) {
    double acc = 0.0;
    GRID_STRIDE(i, n) {
        const double v = psi[i];
        y[i] = 0.0; r[i] = v; p[i] = v;
        acc = fma(v, v, acc);
    }
    block_partial(acc, part);
}

// step s: pq = p^T q (q = (H - sigma) p); breakdown when pq <= 0 or not finite;
// else gamma = rr_s / pq, y += gamma p, r -= gamma q, partial of r^T r
__global__ void __launch_bounds__(kVecBlock) k_cg_xr(int64_t n, int s, double* y, double* r, const double* p,
                                                     const double* q, const double* part, int G, const double* rr,
                                                     const int* cgstop, int* cgbrk, double* part2) {
    if (cgstop[s]) return;
    __shared__ double s_g;
    const double pq = sum_partials(part, G);
    const bool brk = !(pq > 0.0) || !isfinite(pq);
    if (lead()) cgbrk[s] = brk;
    if (brk) return;
    if (threadIdx.x == 0) s_g = rr[s] / pq;   // one thread: divisions are long FP64 chains
    __syncthreads();
    const double g = s_g;
    double acc = 0.0;
    GRID_STRIDE(i, n) {
        y[i] = fma(g, p[i], y[i]);
        const double ri = fma(-g, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    }
    block_partial(acc, part2);
}

// rr_{s+1} = sum(part2); p = r + (rr_{s+1} / rr_s) p; the solve ends after
// step s on a breakdown or when rr_{s+1} <= (1e-10)^2 rr_0
__global__ void __launch_bounds__(kVecBlock) k_cg_p(int64_t n, int s, const double* r, double* p, const double* part2,
                                                    int G, double* rr, int* cgstop, const int* cgbrk) {
    if (cgstop[s] || cgbrk[s]) {
        if (lead()) cgstop[s + 1] = 1;
        return;
    }
    __shared__ double s_be;
    const double rn = sum_partials(part2, G);
    if (threadIdx.x == 0) {   // one thread: divisions are long FP64 chains
        s_be = rn / rr[s];
        if (blockIdx.x == 0) {
            rr[s + 1] = rn;
            cgstop[s + 1] = !(rn > kCgRtol * kCgRtol * rr[0]);
        }
    }
    __syncthreads();
    const double be = s_be;
    GRID_STRIDE(i, n) p[i] = fma(be, p[i], r[i]);
}

// ---- Krylov subspace diagonalisation (Sec. III.B) ----

// P[m][j] = c_m^T v_j for unit projections c_m = e_{idx[m]}
__global__ void k_proj_unit(int M, const int64_t* idx, const double* v, double* P, int nu, int j, const int* stop) {
    if (stop[j]) return;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) P[(size_t)m * nu + j] = v[idx[m]];
}

// partials of c_m^T v for dense projections C[M][n], part[m * G + block]
__global__ void __launch_bounds__(kVecBlock) k_proj_dense(int64_t n, int M, const double* C, const double* v,
                                                          double* part, int G, const int* stop, int j) {
    if (stop[j]) return;
    for (int m = 0; m < M; ++m) {
        double acc = 0.0;
        GRID_STRIDE(i, n) acc = fma(C[(size_t)m * n + i], v[i], acc);
        block_partial(acc, part + (size_t)m * G);
        __syncthreads();
    }
}

// one block per projection: P[m][j] = sum of its partials
__global__ void __launch_bounds__(kVecBlock) k_proj_fin(const double* part, int G, double* P, int nu, int j,
                                                        const int* stop) {
    if (stop[j]) return;
    const double s = sum_partials(part + (size_t)blockIdx.x * G, G);
    if (threadIdx.x == 0) P[(size_t)blockIdx.x * nu + j] = s;
}

// eigenvalue q (ascending) of T, one block of 32 threads each, of which 8
// lanes run a multisection on the Sturm count inside the Gershgorin interval
// (8 points per round, each lane counting at one point), keeping "fewer than
// q + 1 eigenvalues below lo, at least q + 1 below hi".  Eight active lanes
// issue an FP64 warp instruction in a quarter of the time of 32 on this
// GPU's narrow FP64 pipe, which more than pays for the extra rounds.
constexpr int kMsLanes = 8;
// The post-processing kernels below also serve several recursions at once:
// recursion y = blockIdx.y finds its arrays `stride` elements after the
// previous one's (all strides 0 with one recursion).
struct TriStride {
    int64_t tri;     // alpha, beta, ev: nu
    int64_t scale;   // the scale value
    int64_t S;       // eigenvectors: nu * nu
    int64_t work;    // 5 nu * nu
    int64_t PW;      // projections and weights: nproj * nu
    int64_t G;       // nproj * nshift
    int64_t bn;      // ||b||
};

__global__ void k_tri_evals(const int* kdim, const double* alpha, const double* beta, double* ev, double* scale_out,
                            TriStride ys) {
    __shared__ double s_a[kMaxLanczos], s_b2[kMaxLanczos];
    const int y = blockIdx.y;
    kdim += y; alpha += y * ys.tri; beta += y * ys.tri; ev += y * ys.tri;
    if (scale_out) scale_out += y * ys.scale;
    const int k = *kdim;
    const int lane = threadIdx.x;
    const int q = blockIdx.x;
    stage_tri(alpha, beta, k, s_a, s_b2);
    if (lane >= kMsLanes) return;
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i + 1 < k ? fabs(beta[i]) : 0.0);
        lo = fmin(lo, alpha[i] - r);
        hi = fmax(hi, alpha[i] + r);
    }
    const double scale = fmax(fmax(fabs(lo), fabs(hi)), 1e-300);
    if (q == 0 && lane == 0 && scale_out) *scale_out = scale;
    if (q >= k) return;
    const double eps = 2.220446049250313e-16;
    const double pivmin = eps * scale * 1e-3 + 1e-300;
    lo -= 2.0 * eps * scale + pivmin;
    hi += 2.0 * eps * scale + pivmin;
    constexpr unsigned kMask = (1u << kMsLanes) - 1u;
    for (int it = 0; it < 96 && hi - lo > 2.0 * eps * fmax(fabs(lo), fabs(hi)) + pivmin; ++it) {
        const double x = lo + (hi - lo) * ((double)(lane + 1) / (double)(kMsLanes + 1));
        const unsigned above = __ballot_sync(kMask, tri_count_below(s_a, s_b2, k, x, pivmin) >= q + 1);
        const int f = above ? __ffs(above) - 1 : kMsLanes;
        const double xf = __shfl_sync(kMask, x, f < kMsLanes ? f : kMsLanes - 1);
        const double xp = __shfl_sync(kMask, x, f > 0 ? f - 1 : 0);
        if (f == kMsLanes) lo = xf;
        else { hi = xf; if (f > 0) lo = xp; }
    }
    if (lane == 0) ev[q] = 0.5 * (lo + hi);
}

// eigenvectors of T (rows of S, S[q][i]): inverse iteration at each
// eigenvalue with T - e_q factorised by Gaussian elimination with partial
// pivoting.  Eigenvalues closer than 1e-3 ||T|| to their neighbour form a
// cluster (the ghost copies of converged eigenvalues that the Lanczos
// recursion produces without reorthogonalization come in such clusters);
// one thread takes a whole cluster, in ascending order, and orthogonalises
// each iterate against the cluster's earlier vectors.  Clusters are
// independent, one thread each (the thread of the cluster's first
// eigenvalue); `work` holds 5 k doubles per thread.
__global__ void k_tri_evecs(const int* kdim, const double* alpha, const double* beta, const double* ev,
                            const double* scale_p, double* S, double* work, TriStride ys) {
    const int y = blockIdx.y;
    kdim += y; alpha += y * ys.tri; beta += y * ys.tri; ev += y * ys.tri;
    scale_p += y * ys.scale; S += y * ys.S; work += y * ys.work;
    const int k = *kdim;
    const int q0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (q0 >= k) return;
    const double scale = *scale_p;
    const double gap = 1e-3 * scale;
    if (q0 > 0 && ev[q0] - ev[q0 - 1] <= gap) return;          // not the first of its cluster
    const double eps = 2.220446049250313e-16;
    const double tiny = eps * scale + 1e-280;
    double* U0 = work + (size_t)q0 * 5 * k;   // reciprocal of the pivot after the factorisation
    double* U1 = U0 + k;
    double* U2 = U0 + 2 * k;
    double* l = U0 + 3 * k;
    double* sw = U0 + 4 * k;
    for (int q = q0; q < k && (q == q0 || ev[q] - ev[q - 1] <= gap); ++q) {
        // perturb a repeated shift slightly so that the factorisation differs
        const double th = ev[q] + (q - q0) * 10.0 * eps * scale;
        double r0 = alpha[0] - th, r1 = k > 1 ? beta[0] : 0.0, r2 = 0.0;
        for (int i = 0; i + 1 < k; ++i) {
            const double c = beta[i];
            const double d1 = alpha[i + 1] - th, d2 = i + 2 < k ? beta[i + 1] : 0.0;
            double piv;
            if (fabs(r0) >= fabs(c)) {
                const double m = r0 != 0.0 ? c / r0 : 0.0;
                piv = r0; U1[i] = r1; U2[i] = r2; l[i] = m; sw[i] = 0.0;
                r0 = d1 - m * r1; r1 = d2 - m * r2; r2 = 0.0;
            } else {
                const double m = r0 / c;
                piv = c; U1[i] = d1; U2[i] = d2; l[i] = m; sw[i] = 1.0;
                const double n0 = r1 - m * d1, n1 = r2 - m * d2;
                r0 = n0; r1 = n1; r2 = 0.0;
            }
            if (fabs(piv) < tiny) piv = piv < 0.0 ? -tiny : tiny;
            U0[i] = 1.0 / piv;
        }
        U0[k - 1] = 1.0 / (fabs(r0) < tiny ? (r0 < 0.0 ? -tiny : tiny) : r0);
        double* s = S + (size_t)q * k;
        for (int i = 0; i < k; ++i) s[i] = 1.0 + (double)(((i + 3 * q) * 7919) % 13) / 13.0;
        for (int rep = 0; rep < 3; ++rep) {
            for (int i = 0; i + 1 < k; ++i) {
                if (sw[i] != 0.0) { const double t = s[i]; s[i] = s[i + 1]; s[i + 1] = t; }
                s[i + 1] -= l[i] * s[i];
            }
            for (int i = k - 1; i >= 0; --i) {
                double v = s[i];
                if (i + 1 < k) v -= U1[i] * s[i + 1];
                if (i + 2 < k) v -= U2[i] * s[i + 2];
                s[i] = v * U0[i];
            }
            double mx = 0.0;
            for (int i = 0; i < k; ++i) mx = fmax(mx, fabs(s[i]));
            if (!(mx > 0.0) || !isfinite(mx)) break;
            const double imx = 1.0 / mx;
            for (int i = 0; i < k; ++i) s[i] *= imx;
            for (int p = q0; p < q; ++p) {          // Gram-Schmidt against the cluster
                const double* sp = S + (size_t)p * k;
                double dot = 0.0;
                for (int i = 0; i < k; ++i) dot += sp[i] * s[i];
                for (int i = 0; i < k; ++i) s[i] -= dot * sp[i];
            }
            double nr = 0.0;
            for (int i = 0; i < k; ++i) nr += s[i] * s[i];
            if (!(nr > 0.0)) break;
            const double inr = 1.0 / sqrt(nr);
            for (int i = 0; i < k; ++i) s[i] *= inr;
        }
    }
}

// weight[m][q] = (c_m^T w_q)(w_q^T b) = (sum_j S[q][j] P[m][j]) ||b|| S[q][0]; one thread per (m, q)
__global__ void k_krylov_weight(const int* kdim, int M, int nu, const double* S, const double* P,
                                const double* bnorm, double* W, TriStride ys) {
    const int y = blockIdx.y;
    kdim += y; S += y * ys.S; P += y * ys.PW; bnorm += y * ys.bn; W += y * ys.PW;
    const int k = *kdim;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M * k) return;
    const int m = t / k, q = t % k;
    const double* s = S + (size_t)q * k;
    const double* p = P + (size_t)m * nu;
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = fma(s[j], p[j], acc);
    W[(size_t)m * nu + q] = acc * (*bnorm) * s[0];
}

// G[m][kk] = sum_q weight[m][q] / (z_kk - e_q); one thread per (m, kk)
__global__ void k_krylov_g(const int* kdim, int M, int nu, int K, const double* ev, const double* W,
                           const double2* z, double2* G, TriStride ys) {
    const int y = blockIdx.y;
    kdim += y; ev += y * ys.tri; W += y * ys.PW; G += y * ys.G;
    const int k = *kdim;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M * K) return;
    const int m = t / K, kk = t % K;
    const double2 zz = z[kk];
    double gr = 0.0, gi = 0.0;
    for (int q = 0; q < k; ++q) {
        const double dr = zz.x - ev[q], di = zz.y;
        const double w = W[(size_t)m * nu + q] / fma(dr, dr, di * di);   // w / |z - e|^2
        gr = fma(w, dr, gr);
        gi = fma(-w, di, gi);
    }
    G[t] = make_double2(gr, gi);
}

#undef GRID_STRIDE

// Device scalars of one call, carved from one allocation.
struct GroundScalars {
    double* alpha;    // [m]
    double* beta;     // [m]
    double* tnorm;    // [m]
    double* s;        // [m]  eigenvector of T
    double* work;     // [5 m]
    double* scal;     // [4]: theta of T, E, res, spare
    double* part;     // [G]
    double* part2;    // [G]
    double* rr;       // [cg + 1]
    int* stop;        // [m + 1]
    int* kdim;        // [1]
    int* ok;          // [1]
    int* cgstop;      // [cg + 1]
    int* cgbrk;       // [cg]
};

}  // namespace

// Blocks of the operator launch (= its partials): the Hubbard operator is
// FP64 bound and takes the vector grid; the CSR operator is bound by its
// dependent index -> gather loads and takes one 8-lane group per row (up to
// 32 blocks per SM), so every row's loads are in flight at once.
static bool use_bsr(const scocg_ctx* h) {
    return h->kind == HandleKind::kCsr && h->bsr_ok && h->opts.layout != 1 && h->d_bval64 && h->d_unit_off &&
           h->d_bcol;
}

static int apply_grid(const scocg_ctx* h, int G) {
    if (h->kind == HandleKind::kHubbard) return G;
    const int64_t want = use_bsr(h) ? (h->nunits_bsr * 32 + kVecBlock - 1) / kVecBlock
                                    : (h->n * 8 + kVecBlock - 1) / kVecBlock;
    return (int)std::max<int64_t>(G, std::min<int64_t>(want, 32LL * h->num_sms));
}

// Real FP64 operator of the handle: y = (H - sigma) x - beta x_prev, partial of x^T y.
static cudaError_t hx(scocg_ctx* h, const double* x, double* y, const double* xprev, const double* beta,
                      double sigma, const int* skip, double* part, int G) {
    if (h->kind == HandleKind::kHubbard) return hubbard_hx(h->hub, x, y, xprev, beta, sigma, skip, part, G, h->stream);
    if (use_bsr(h)) {
        k_bsr4_hx<<<G, kVecBlock, 0, h->stream>>>(h->nunits_bsr, h->d_unit_off, h->d_bcol, h->d_bval64, h->n, x, y,
                                                   xprev, beta, sigma, skip, part);
        return cudaGetLastError();
    }
    k_csr_hx<<<G, kVecBlock, 0, h->stream>>>(h->n, h->d_rowptr, h->d_col, h->d_val64, x, y, xprev, beta, sigma, skip,
                                              part);
    return cudaGetLastError();
}

// Algorithmic bytes of one Lanczos step: H once (CSR: int32 index + FP64 value
// per entry and the row pointers; Hubbard: the hop tables) plus the vector
// passes: apply (read v_j, v_{j-1}, write w, gather v_j), ortho (read v_j, w,
// write w), next (read w, write v_{j+1}) = 8 passes of 8 bytes.
static double lanczos_step_bytes(const scocg_ctx* h) {
    const double hb = h->kind == HandleKind::kHubbard ? h->hub.table_bytes
                                                      : 12.0 * (double)h->nnz + 4.0 * (double)(h->n + 1);
    return hb + 8.0 * 8.0 * (double)h->n;
}

}  // namespace scocg

using namespace scocg;

extern "C" int scocg_ground_state(scocg_handle h, const double* v0, double* psi_out, int m, int cg_steps,
                                  int max_cycles, double tol, double* energy, scocg_ground_info* info) {
    if (!h || !v0 || !psi_out || !energy || m < 2 || m > kMaxLanczos || cg_steps < 0 || cg_steps > 1000000 ||
        max_cycles < 1 || !(tol >= 0.0) || !std::isfinite(tol))
        return SCOCG_ERR_INVALID;
    if (h->kind == HandleKind::kCsr && !h->d_val64) return SCOCG_ERR_INVALID;
    const int64_t n = h->n;
    if (n < 1) return SCOCG_ERR_INVALID;
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>((n + kVecBlock - 1) / kVecBlock, 8LL * h->num_sms));
    const int mm = (int)std::min<int64_t>(m, n);   // at most n Lanczos vectors are independent
    const int Gh = apply_grid(h, G);               // blocks (partials) of the operator launches
    // device memory: V[mm][n], w, psi, y, r, p and the scalars
    Carver cv{nullptr, 0};
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            void* base = nullptr;
            if (cudaMalloc(&base, cv.off) != cudaSuccess) { cudaGetLastError(); return SCOCG_ERR_OOM; }
            cv = Carver{static_cast<char*>(base), 0};
        }
        cv.take(sizeof(double) * (size_t)mm * n);
        for (int v = 0; v < 5; ++v) cv.take(sizeof(double) * n);
        cv.take(sizeof(double) * (9 * (size_t)mm + 4 + 2 * (size_t)Gh + cg_steps + 1));
        cv.take(sizeof(int) * ((size_t)mm + 3 + 2 * (size_t)cg_steps + 1));
    }
    char* base = cv.base;
    cv.off = 0;
    double* V = (double*)cv.take(sizeof(double) * (size_t)mm * n);
    double* w = (double*)cv.take(sizeof(double) * n);
    double* psi = (double*)cv.take(sizeof(double) * n);
    double* y = (double*)cv.take(sizeof(double) * n);
    double* r = (double*)cv.take(sizeof(double) * n);
    double* p = (double*)cv.take(sizeof(double) * n);
    GroundScalars S;
    {
        double* d = (double*)cv.take(sizeof(double) * (9 * (size_t)mm + 4 + 2 * (size_t)Gh + cg_steps + 1));
        S.alpha = d; S.beta = d + mm; S.tnorm = d + 2 * mm; S.s = d + 3 * mm; S.work = d + 4 * mm;
        S.scal = d + 9 * mm; S.part = S.scal + 4; S.part2 = S.part + Gh; S.rr = S.part2 + Gh;
        int* q = (int*)cv.take(sizeof(int) * ((size_t)mm + 3 + 2 * (size_t)cg_steps + 1));
        S.stop = q; S.kdim = q + mm + 1; S.ok = S.kdim + 1; S.cgstop = S.ok + 1; S.cgbrk = S.cgstop + cg_steps + 1;
    }
    cudaStream_t st = h->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(psi, v0, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    int status = SCOCG_NOT_CONVERGED;
    long long lanczos_total = 0, cg_total = 0;
    int cycles = 0;
    double E = NAN, res = NAN;
    std::vector<int> host_stop(cg_steps + 1);
    for (int cyc = 0; cyc < max_cycles && e == cudaSuccess; ++cyc) {
        ++cycles;
        // v_0 = psi / ||psi||
        k_norm_part<<<G, kVecBlock, 0, st>>>(n, psi, S.part);
        k_scale_to<<<G, kVecBlock, 0, st>>>(n, psi, V, S.part, G, S.ok);
        if (cyc == 0) {   // a zero or non-finite start vector is an invalid argument
            int ok = 0;
            e = cudaMemcpyAsync(&ok, S.ok, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess && !ok) { status = SCOCG_ERR_INVALID; break; }
            if (e != cudaSuccess) break;
        }
        e = cudaMemsetAsync(S.stop, 0, sizeof(int) * (mm + 1), st);
        const int mm_v = mm;
        if (e == cudaSuccess) e = cudaMemcpyAsync(S.kdim, &mm_v, sizeof(int), cudaMemcpyHostToDevice, st);
        for (int j = 0; j < mm && e == cudaSuccess; ++j) {
            const double* vj = V + (size_t)j * n;
            e = hx(h, vj, w, j ? vj - n : nullptr, j ? S.beta + j - 1 : nullptr, 0.0, S.stop + j, S.part, Gh);
            if (e != cudaSuccess) break;
            k_lz_ortho<<<G, kVecBlock, 0, st>>>(n, j, vj, w, S.part, Gh, S.stop, S.alpha, S.part2);
            k_lz_next<<<G, kVecBlock, 0, st>>>(n, j, mm, w, j + 1 < mm ? V + (size_t)(j + 1) * n : w, S.part2, G,
                                               S.alpha, S.beta, S.tnorm, S.stop, S.kdim);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) break;
        k_tri_lowest<<<1, 32, 0, st>>>(S.kdim, S.alpha, S.beta, S.s, S.work, S.scal);
        k_ritz<<<G, kVecBlock, 0, st>>>(n, S.kdim, S.s, V, w, S.part);
        k_scale_to<<<G, kVecBlock, 0, st>>>(n, w, psi, S.part, G, S.ok);
        e = hx(h, psi, w, nullptr, nullptr, 0.0, nullptr, S.part, Gh);
        if (e != cudaSuccess) break;
        k_resid<<<G, kVecBlock, 0, st>>>(n, psi, w, S.part, Gh, S.part2, S.scal + 1);
        k_sum_store<<<1, kVecBlock, 0, st>>>(S.part2, G, S.scal + 2, 1);
        double sc[3];
        int kd = 0;
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(sc, S.scal, sizeof(sc), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&kd, S.kdim, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        lanczos_total += kd;
        E = sc[1];
        res = sc[2];
        if (!std::isfinite(E) || !std::isfinite(res)) { status = SCOCG_ERR_BREAKDOWN; break; }
        if (res <= tol) { status = SCOCG_OK; break; }
        if (cg_steps == 0 || cyc + 1 == max_cycles) continue;
        // inverse iteration: CG on (H - sigma) y = psi
        const double sigma = E - res;
        k_cg_init<<<G, kVecBlock, 0, st>>>(n, psi, y, r, p, S.part);
        k_sum_store<<<1, kVecBlock, 0, st>>>(S.part, G, S.rr, 0);
        e = cudaMemsetAsync(S.cgstop, 0, sizeof(int) * (2 * (size_t)cg_steps + 1), st);
        for (int s = 0; s < cg_steps && e == cudaSuccess; ++s) {
            e = hx(h, p, w, nullptr, nullptr, sigma, S.cgstop + s, S.part, Gh);
            if (e != cudaSuccess) break;
            k_cg_xr<<<G, kVecBlock, 0, st>>>(n, s, y, r, p, w, S.part, Gh, S.rr, S.cgstop, S.cgbrk, S.part2);
            k_cg_p<<<G, kVecBlock, 0, st>>>(n, s, r, p, S.part2, G, S.rr, S.cgstop, S.cgbrk);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) break;
        k_norm_part<<<G, kVecBlock, 0, st>>>(n, y, S.part);
        k_scale_to<<<G, kVecBlock, 0, st>>>(n, y, psi, S.part, G, S.ok);   // psi kept if y = 0
        e = cudaMemcpyAsync(host_stop.data(), S.cgstop, sizeof(int) * (cg_steps + 1), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            int taken = 0;
            while (taken < cg_steps && !host_stop[taken]) ++taken;
            cg_total += taken;
        }
    }
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(psi_out, psi, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(base);
    if (e != cudaSuccess) return cuda_status(e);
    if (status == SCOCG_ERR_INVALID) return status;
    *energy = E;
    if (info) {
        info->cycles = cycles;
        info->lanczos_steps = lanczos_total;
        info->cg_steps = cg_total;
        info->residual = res;
        info->seconds = ms * 1e-3;
        info->bytes_per_step = lanczos_step_bytes(h);
    }
    return status;
}

extern "C" int scocg_krylov_sd(scocg_handle h, const double* b, int nu, const scocg_c128* shifts, int nshift,
                               const int64_t* proj_idx, const double* proj_vec, int nproj, scocg_c128* G_out,
                               double* ritz, double* weight, int* nu_used, double* seconds) {
    if (!h || !b || nu < 1 || nu > kMaxLanczos || !shifts || nshift < 1 || nshift > (1 << 20) || nproj < 1 ||
        nproj > 64 || (!proj_idx) == (!proj_vec) || !G_out)
        return SCOCG_ERR_INVALID;
    if (h->kind == HandleKind::kCsr && !h->d_val64) return SCOCG_ERR_INVALID;
    const int64_t n = h->n;
    if (n < 1) return SCOCG_ERR_INVALID;
    for (int k = 0; k < nshift; ++k)
        if (!std::isfinite(shifts[k].re) || !std::isfinite(shifts[k].im)) return SCOCG_ERR_INVALID;
    if (proj_idx)
        for (int m = 0; m < nproj; ++m)
            if (proj_idx[m] < 0 || proj_idx[m] >= n) return SCOCG_ERR_INVALID;
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>((n + kVecBlock - 1) / kVecBlock, 8LL * h->num_sms));
    const int M = nproj, K = nshift;
    int Gh = apply_grid(h, G);
    // one cooperative launch for the whole recursion when the layout allows it
    int Gp = 0;
    if (use_bsr(h) && proj_idx) {
        int nb = 0;
        // two CTAs per SM: measured faster than the occupancy maximum of three on
        // the 32^3 x 4 matrix (7.9 vs 9.2 ms per 200 steps; the grid barriers and
        // the block sums grow with the CTA count), and than one (8.8 ms)
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_krylov_lanczos, kVecBlock, 0) == cudaSuccess && nb > 0)
            Gp = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::min(nb, 2) * h->num_sms,
                                                             (h->nunits_bsr * 32 + kVecBlock - 1) / kVecBlock));
        cudaGetLastError();
        if (Gp > 0 && h->opts.grid > 0) Gp = std::min(Gp, h->opts.grid);   // the handle's grid option, clamped
        Gh = std::max(Gh, Gp);
    }
    Carver cv{nullptr, 0};
    double *vb[3], *w, *P, *S, *W, *work, *alpha, *beta, *tnorm, *ev, *scal, *part, *part2, *partM;
    int *stop, *kdim;
    int64_t* d_idx;
    double2* d_z;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            void* base = nullptr;
            if (cudaMalloc(&base, cv.off) != cudaSuccess) { cudaGetLastError(); return SCOCG_ERR_OOM; }
            cv = Carver{static_cast<char*>(base), 0};
        }
        for (int v = 0; v < 3; ++v) vb[v] = (double*)cv.take(sizeof(double) * n);
        w = (double*)cv.take(sizeof(double) * n);
        P = (double*)cv.take(sizeof(double) * (size_t)M * nu);
        S = (double*)cv.take(sizeof(double) * (size_t)nu * nu);
        W = (double*)cv.take(sizeof(double) * (size_t)M * nu);
        work = (double*)cv.take(sizeof(double) * 5 * (size_t)nu * nu);
        alpha = (double*)cv.take(sizeof(double) * nu);
        beta = (double*)cv.take(sizeof(double) * nu);
        tnorm = (double*)cv.take(sizeof(double) * nu);
        ev = (double*)cv.take(sizeof(double) * nu);
        scal = (double*)cv.take(sizeof(double) * 4);
        part = (double*)cv.take(sizeof(double) * Gh);
        part2 = (double*)cv.take(sizeof(double) * Gh);
        partM = (double*)cv.take(sizeof(double) * (size_t)M * G);
        stop = (int*)cv.take(sizeof(int) * (nu + 1));
        kdim = (int*)cv.take(sizeof(int));
        d_idx = (int64_t*)cv.take(sizeof(int64_t) * M);
        d_z = (double2*)cv.take(sizeof(double2) * K);
    }
    char* base = cv.base;
    cudaStream_t st = h->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_z, shifts, sizeof(double2) * K, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && proj_idx)
        e = cudaMemcpyAsync(d_idx, proj_idx, sizeof(int64_t) * M, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(stop, 0, sizeof(int) * (nu + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P, 0, sizeof(double) * (size_t)M * nu, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    int status = SCOCG_OK;
    if (e == cudaSuccess) {
        // v_0 = b / ||b||, ||b|| kept for the weights
        k_norm_part<<<G, kVecBlock, 0, st>>>(n, b, part);
        k_sum_store<<<1, kVecBlock, 0, st>>>(part, G, scal, 1);
        k_scale_to<<<G, kVecBlock, 0, st>>>(n, b, vb[0], part, G, kdim);
        int ok = 0;
        e = cudaMemcpyAsync(&ok, kdim, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && !ok) status = SCOCG_ERR_INVALID;
    }
    if (Gp > 0 && e == cudaSuccess && status == SCOCG_OK) {
        KrylovArgs ka;
        ka.n = n; ka.nunits = h->nunits_bsr;
        ka.unit_off = h->d_unit_off; ka.bcol = h->d_bcol; ka.bval = h->d_bval64;
        ka.b = b;
        ka.V[0] = vb[0]; ka.V[1] = vb[1]; ka.W[0] = vb[2]; ka.W[1] = w;
        ka.nu = nu; ka.M = M; ka.idx = d_idx; ka.P = P;
        ka.alpha = alpha; ka.beta = beta; ka.kdim = kdim;
        ka.part_a = part; ka.part_b = part2;
        ka.sync.count = &h->d_ctrl->count;
        ka.sync.status = &h->d_ctrl->status;
        ka.sync.timeout_ns = (uint64_t)(h->opts.timeout_ms * 1e6);
        ka.sync.nctas = Gp;
        e = cudaMemsetAsync(h->d_ctrl, 0, sizeof(Ctrl), st);
        void* args[] = {(void*)&ka};
        if (e == cudaSuccess)
            e = cudaLaunchCooperativeKernel((const void*)k_krylov_lanczos, dim3(Gp), dim3(kVecBlock), args, 0, st);
    }
    for (int j = 0; Gp == 0 && j < nu && e == cudaSuccess && status == SCOCG_OK; ++j) {
        const double* vj = vb[j % 3];
        if (proj_idx) {
            k_proj_unit<<<(M + 63) / 64, 64, 0, st>>>(M, d_idx, vj, P, nu, j, stop);
        } else {
            k_proj_dense<<<G, kVecBlock, 0, st>>>(n, M, proj_vec, vj, partM, G, stop, j);
            k_proj_fin<<<M, kVecBlock, 0, st>>>(partM, G, P, nu, j, stop);
        }
        e = hx(h, vj, w, j ? vb[(j + 2) % 3] : nullptr, j ? beta + j - 1 : nullptr, 0.0, stop + j, part, Gh);
        if (e != cudaSuccess) break;
        k_lz_ortho<<<G, kVecBlock, 0, st>>>(n, j, vj, w, part, Gh, stop, alpha, part2);
        k_lz_next<<<G, kVecBlock, 0, st>>>(n, j, nu, w, vb[(j + 1) % 3], part2, G, alpha, beta, tnorm, stop, kdim);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && status == SCOCG_OK) {
        const TriStride one{};
        k_tri_evals<<<nu, 32, 0, st>>>(kdim, alpha, beta, ev, scal + 1, one);
        k_tri_evecs<<<(nu + 7) / 8, 8, 0, st>>>(kdim, alpha, beta, ev, scal + 1, S, work, one);
        k_krylov_weight<<<(M * nu + 127) / 128, 128, 0, st>>>(kdim, M, nu, S, P, scal, W, one);
        k_krylov_g<<<(M * K + 127) / 128, 128, 0, st>>>(kdim, M, nu, K, ev, W, d_z, (double2*)G_out, one);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess && ritz) e = cudaMemcpyAsync(ritz, ev, sizeof(double) * nu, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && weight)
            e = cudaMemcpyAsync(weight, W, sizeof(double) * (size_t)M * nu, cudaMemcpyDeviceToDevice, st);
        int kd = 0, bar = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&kd, kdim, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && Gp > 0) e = cudaMemcpyAsync(&bar, &h->d_ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && bar < 0) status = bar;   // a grid barrier gave up (SCOCG_ERR_TIMEOUT)
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) {
            if (nu_used) *nu_used = kd;
            if (seconds) *seconds = ms * 1e-3;
        }
    }
    if (e != cudaSuccess) cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(base);
    if (e != cudaSuccess) return cuda_status(e);
    return status;
}

// ---------------------------------------------------------------- several right-hand sides
#ifndef SCOCG_KRSD_CTAS_PER_SM
#define SCOCG_KRSD_CTAS_PER_SM 2
#endif
#ifndef SCOCG_KRSD_DF_CTAS_PER_SM
#define SCOCG_KRSD_DF_CTAS_PER_SM 2   // the compensated recursion measured the same with 2, 4 and 6
#endif
namespace scocg {
namespace {
template <int T>
int krylov_block_grid(const scocg_ctx* h, bool df) {
    int nb = 0;
    const cudaError_t oe = df ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_krylov_block_df<T>, kVecBlock, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_krylov_block<T>, kVecBlock, 0);
    if (oe != cudaSuccess || nb < 1) {
        cudaGetLastError();
        return 0;
    }
    // up to SCOCG_KRSD_CTAS_PER_SM CTAs per SM (two: 39.5 ms for 200 steps of
    // 16 recursions on the 32^3 x 4 matrix, against 45.0 with four and 48.2
    // with eight), at most one warp step of block rows per warp
    const int64_t steps = (h->nunits_bsr * 8 + (kVecBlock / 32) * (32 / T) - 1) / ((kVecBlock / 32) * (32 / T));
    const int per_sm = df ? SCOCG_KRSD_DF_CTAS_PER_SM : SCOCG_KRSD_CTAS_PER_SM;
    int g = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::min(nb, per_sm) * h->num_sms, steps));
    if (h->opts.grid > 0) g = std::min(g, h->opts.grid);
    return g;
}

template <int T>
cudaError_t launch_krylov_block(const KrylovBlockArgs& ka, int grid, cudaStream_t st) {
    void* args[] = {(void*)&ka};
    return cudaLaunchCooperativeKernel((const void*)k_krylov_block<T>, dim3(grid), dim3(kVecBlock), args, 0, st);
}
template <int T>
cudaError_t launch_krylov_block_df(const KrylovBlockDfArgs& ka, int grid, cudaStream_t st) {
    void* args[] = {(void*)&ka};
    return cudaLaunchCooperativeKernel((const void*)k_krylov_block_df<T>, dim3(grid), dim3(kVecBlock), args, 0, st);
}
}  // namespace
}  // namespace scocg

extern "C" int scocg_krylov_sd_multi(scocg_handle h, const double* B, int nrhs, int nu, const scocg_c128* shifts,
                                     int nshift, const int64_t* proj_idx, int nproj, scocg_c128* G_out,
                                     int* nu_used, double* seconds) {
    if (!h || !B || nrhs < 1 || nu < 1 || nu > kMaxLanczos || !shifts || nshift < 1 || nshift > (1 << 20) ||
        !proj_idx || nproj < 1 || nproj > 64 || !G_out)
        return SCOCG_ERR_INVALID;
    const int64_t n = h->n;
    const int M = nproj, K = nshift;
    for (int k = 0; k < K; ++k)
        if (!std::isfinite(shifts[k].re) || !std::isfinite(shifts[k].im)) return SCOCG_ERR_INVALID;
    for (int64_t j = 0; j < (int64_t)nrhs * M; ++j)
        if (proj_idx[j] < 0 || proj_idx[j] >= n) return SCOCG_ERR_INVALID;
    if (!use_bsr(h)) {
        // other layouts: the one-right-hand-side recursion per right-hand side
        double total = 0.0;
        for (int r = 0; r < nrhs; ++r) {
            int used = 0;
            double sec = 0.0;
            const int st = scocg_krylov_sd(h, B + (size_t)r * n, nu, shifts, K, proj_idx + (size_t)r * M, nullptr,
                                           M, G_out + (size_t)r * M * K, nullptr, nullptr, &used, &sec);
            if (st != SCOCG_OK) return st;
            if (nu_used) nu_used[r] = used;
            total += sec;
        }
        if (seconds) *seconds = total;
        return SCOCG_OK;
    }
    const int T = nrhs <= 8 ? 8 : (nrhs <= 16 ? 16 : 32);
    // compensated FP32 recursion for SCOCG_MIXED_DF handles (H's FP32 blocks)
    const bool df = h->opts.precision == SCOCG_MIXED_DF && h->d_bval32;
    const int Gp = T == 8 ? krylov_block_grid<8>(h, df) : T == 16 ? krylov_block_grid<16>(h, df)
                                                         : krylov_block_grid<32>(h, df);
    if (Gp < 1) return SCOCG_ERR_CUDA;
    Carver cv{nullptr, 0};
    double *X0 = nullptr, *vb[4] = {nullptr, nullptr, nullptr, nullptr}, *P = nullptr, *alpha = nullptr,
           *beta = nullptr, *bnorm = nullptr, *pa = nullptr, *pb = nullptr, *S = nullptr, *work = nullptr,
           *ev = nullptr, *W = nullptr, *scal = nullptr;
    int* kdim = nullptr;
    int64_t* d_idx = nullptr;
    double2* d_z = nullptr;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            void* base = nullptr;
            if (cudaMalloc(&base, cv.off) != cudaSuccess) { cudaGetLastError(); return SCOCG_ERR_OOM; }
            cv = Carver{static_cast<char*>(base), 0};
        }
        X0 = (double*)cv.take(sizeof(double) * (size_t)n * T);
        for (int v = 0; v < 4; ++v) vb[v] = (double*)cv.take(sizeof(double) * (size_t)n * T);
        P = (double*)cv.take(sizeof(double) * (size_t)T * M * nu);
        alpha = (double*)cv.take(sizeof(double) * (size_t)T * nu);
        beta = (double*)cv.take(sizeof(double) * (size_t)T * nu);
        bnorm = (double*)cv.take(sizeof(double) * T);
        kdim = (int*)cv.take(sizeof(int) * T);
        pa = (double*)cv.take(sizeof(double) * (size_t)T * Gp);
        pb = (double*)cv.take(sizeof(double) * (size_t)T * Gp);
        d_idx = (int64_t*)cv.take(sizeof(int64_t) * (size_t)T * M);
        d_z = (double2*)cv.take(sizeof(double2) * K);
        // post-processing scratch, per slot
        S = (double*)cv.take(sizeof(double) * (size_t)T * nu * nu);
        work = (double*)cv.take(sizeof(double) * 5 * (size_t)T * nu * nu);
        ev = (double*)cv.take(sizeof(double) * (size_t)T * nu);
        W = (double*)cv.take(sizeof(double) * (size_t)T * M * nu);
        scal = (double*)cv.take(sizeof(double) * 4 * T);
    }
    char* base = cv.base;
    cudaStream_t st = h->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_z, shifts, sizeof(double2) * K, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    int status = SCOCG_OK;
    std::vector<int> kd(T);
    std::vector<double> bn(T);
    std::vector<int64_t> idx_tile((size_t)T * M);
    for (int r0 = 0; r0 < nrhs && e == cudaSuccess && status == SCOCG_OK; r0 += T) {
        const int ns = std::min(T, nrhs - r0);
        for (int t = 0; t < T; ++t)
            for (int m = 0; m < M; ++m) idx_tile[(size_t)t * M + m] = t < ns ? proj_idx[(size_t)(r0 + t) * M + m] : 0;
        e = cudaMemcpyAsync(d_idx, idx_tile.data(), sizeof(int64_t) * idx_tile.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            if (df)
                k_to_slots_df<<<(unsigned)((n * T + 255) / 256), 256, 0, st>>>(n, T, ns, B + (size_t)r0 * n,
                                                                               (float2*)X0);
            else
                k_to_slots<<<(unsigned)((n * T + 255) / 256), 256, 0, st>>>(n, T, ns, B + (size_t)r0 * n, X0);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(P, 0, sizeof(double) * (size_t)T * M * nu, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->d_ctrl, 0, sizeof(Ctrl), st);
        if (e != cudaSuccess) break;
        KrylovBlockArgs ka;
        ka.n = n; ka.nunits = h->nunits_bsr;
        ka.unit_off = h->d_unit_off; ka.bcol = h->d_bcol; ka.bval = h->d_bval64;
        ka.B = X0;
        ka.V[0] = vb[0]; ka.V[1] = vb[1]; ka.W[0] = vb[2]; ka.W[1] = vb[3];
        ka.nu = nu; ka.M = M; ka.nslot = ns;
        ka.idx = d_idx; ka.P = P; ka.alpha = alpha; ka.beta = beta; ka.bnorm = bnorm; ka.kdim = kdim;
        ka.part_a = pa; ka.part_b = pb;
        ka.sync.count = &h->d_ctrl->count;
        ka.sync.status = &h->d_ctrl->status;
        ka.sync.timeout_ns = (uint64_t)(h->opts.timeout_ms * 1e6);
        ka.sync.nctas = Gp;
        if (df) {
            KrylovBlockDfArgs kd2;
            kd2.n = n; kd2.nunits = h->nunits_bsr;
            kd2.unit_off = h->d_unit_off; kd2.bcol = h->d_bcol; kd2.bval = h->d_bval32;
            kd2.B = (const float2*)X0;
            kd2.V[0] = (float2*)vb[0]; kd2.V[1] = (float2*)vb[1]; kd2.W[0] = (float2*)vb[2]; kd2.W[1] = (float2*)vb[3];
            kd2.nu = nu; kd2.M = M; kd2.nslot = ns;
            kd2.idx = d_idx; kd2.P = P; kd2.alpha = alpha; kd2.beta = beta; kd2.bnorm = bnorm; kd2.kdim = kdim;
            kd2.part_a = pa; kd2.part_b = pb;
            kd2.sync = ka.sync;
            e = T == 8 ? launch_krylov_block_df<8>(kd2, Gp, st)
                : T == 16 ? launch_krylov_block_df<16>(kd2, Gp, st) : launch_krylov_block_df<32>(kd2, Gp, st);
        } else {
            e = T == 8 ? launch_krylov_block<8>(ka, Gp, st)
                : T == 16 ? launch_krylov_block<16>(ka, Gp, st) : launch_krylov_block<32>(ka, Gp, st);
        }
        int bar = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(kd.data(), kdim, sizeof(int) * T, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bn.data(), bnorm, sizeof(double) * T, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bar, &h->d_ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        if (bar < 0) { status = bar; break; }   // a grid barrier gave up (SCOCG_ERR_TIMEOUT)
        for (int t = 0; t < ns; ++t)
            if (!(bn[t] > 0.0)) status = SCOCG_ERR_INVALID;   // b = 0
        if (status != SCOCG_OK) break;
        // the tridiagonal eigenproblems, weights and G of all ns recursions together
        const TriStride ys{nu, 4, (int64_t)nu * nu, 5LL * nu * nu, (int64_t)M * nu, (int64_t)M * K, 1};
        k_tri_evals<<<dim3(nu, ns), 32, 0, st>>>(kdim, alpha, beta, ev, scal + 1, ys);
        k_tri_evecs<<<dim3((nu + 7) / 8, ns), 8, 0, st>>>(kdim, alpha, beta, ev, scal + 1, S, work, ys);
        k_krylov_weight<<<dim3((M * nu + 127) / 128, ns), 128, 0, st>>>(kdim, M, nu, S, P, bnorm, W, ys);
        k_krylov_g<<<dim3((M * K + 127) / 128, ns), 128, 0, st>>>(kdim, M, nu, K, ev, W, d_z,
                                                                 (double2*)(G_out + (size_t)r0 * M * K), ys);
        e = cudaGetLastError();
        for (int t = 0; t < ns; ++t)
            if (nu_used) nu_used[r0 + t] = kd[t];
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && seconds) *seconds = ms * 1e-3;
    if (e != cudaSuccess) cudaStreamSynchronize(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(base);
    if (e != cudaSuccess) return cuda_status(e);
    return status;
}
