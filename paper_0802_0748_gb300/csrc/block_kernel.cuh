// Persistent multi-right-hand-side shifted-COCG kernel ("block" mode).
//
// T right-hand sides advance together in T column slots, each slot with its
// own seed COCG scalars (Sec. III.C), shifts and per-shift recurrences, and all
// slots share every read of H: the seed apply becomes a sparse-times-dense
// product over vectors stored row-major [n][T] (a row's T entries are one
// coalesced line).  Per seed iteration (A_c = z_{s,c} I - H for slot c):
//   phase A  q_c = A_c r_c + beta_c q_c, partial r_c^T q_c          -> barrier
//   decide   alpha_c = rho_c / (r_c^T q_c); a slot whose shifts have all
//            converged (or that failed) writes its outputs and is refilled
//            with the next right-hand side (or left empty)
//   phase B  r_c -= alpha_c q_c; a refilled slot loads r_c = b, q_c = 0;
//            partials r^T r, ||r||^2, ||b||^2                       -> barrier
//   phase C  per (slot, shift) pair: the pi three-term recurrence, projected
//            P and X, residual and freezing (or the pair's initial state
//            for a refilled slot); then per-slot seed switching.
// Slots therefore stay busy while right-hand sides converge at different
// iteration counts.  Projections are unit vectors, per right-hand side.
#pragma once
#include <climits>

#include "solver_kernel.cuh"

namespace scocg {

constexpr int kNvA = 4;          // per-slot partials of phase A: r^T q (2), active, bad
constexpr int kNvB = 4;          // phase B: r^T r (2), ||r||^2, ||b||^2
constexpr int kNvC = 10;         // switching: active, |1/pi| key, arg, bad, pi_prev, pi_cur, alpha_k (2 each)
enum : int { kSlotEmpty = 0, kSlotRun = 1, kSlotFresh = 2 };

template <typename R>
struct BlockArgs {
    using V = typename Vec<R>::T;
    using W = typename ValT<R>::T;
    int64_t n;
    int64_t nnz;
    const int* rowptr;           // int32 CSR of H
    const int* col;
    const W* val;
    V* r;                        // [n][T]
    V* q;                        // [n][T]
    const double2* b;            // rhs, complex128 [nrhs][n]
    int nrhs;
    const int64_t* cidx;         // [nrhs][nproj] unit projections
    int nproj;
    int K;
    const double2* z;            // [K]
    int seed0;                   // initial seed of every right-hand side
    int allow_switch;
    double tol;
    int max_iter;
    // (slot, shift) pair state, pair p = slot * K + k
    double2* pi_prev;
    double2* pi_cur;
    double2* sigma;
    double2* alpha_k;
    double2* inv_cur;
    double2* P;                  // [T][K][nproj]
    double2* X;                  // [T][K][nproj]
    int* frozen;
    int* iters;
    double* resid;               // squared residual estimates
    // per right-hand side outputs
    double2* G;                  // [nrhs][nproj][K]
    int* out_iters;              // [nrhs][K] freeze iteration
    double* out_resid;           // [nrhs][K] squared residual estimate
    int* out_info;               // [nrhs][4]: status, seed iterations, switches, final seed
    // per-CTA partials, value-major: part[v * grid + cta]
    double* partA;               // [kNvA * T][grid]
    double* partB;               // [kNvB * T][grid]
    double* partC;               // [kNvC * T][grid]
    GridSync sync;
    SolveStats* stats;
    unsigned long long* dbg;
    // 4x4-blocked sliced ELL of H (unit_off null: the CSR apply above)
    const int* unit_off;
    const int* bcol;
    const W* bval;                  // row-major 4x4 blocks
    int64_t nslots;
    unsigned long long* phase_ns;   // phase-timer builds: [grid][8] accumulated ns
    double* res;                    // [max(kNvA, kNvB) * T] sums published by grid_reduce
};

template <int T>
struct BlockShared {
    double2 zs[T], alpha[T], alpha_prev[T], beta_prev[T], rho[T], rho_new[T], t2[T];
    double2 sw_inv1[T], sw_ca[T], sw_cb[T], sw_pin[T], sw_pin1[T], sw_alpha[T];
    double bnorm[T], rn_b2[T];
    double2 cr_cur[T * kMaxProjB], cr_next[T * kMaxProjB];
    unsigned long long key[T];
    long long siters[T];
    int state[T], rhs[T], seed[T], n[T], fin[T], nsw[T], pend[T], sw[T], s2[T], arg[T];
    int cnt[T], bad[T];
    int next_rhs, any_live;
    double red[kNvB * T > kNvA * T ? kNvB * T : kNvA * T];
    double scratch[kWarps * T * 4];
};

// Sum over the lanes of a warp that serve the same slot (lanes l, l + T, ...).
template <int T> __device__ __forceinline__ double col_sum(double v) {
#pragma unroll
    for (int o = T; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int T> __device__ __forceinline__ float col_sum(float v) {
#pragma unroll
    for (int o = T; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int T> __device__ __forceinline__ dfs col_sum(dfs v) {
#pragma unroll
    for (int o = T; o < 32; o <<= 1) {
        dfs w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = df_add(v, w);
    }
    return v;
}

// Per-slot CTA partials: value j of slot c (this lane's slot) goes to
// part[(c * NVS + j) * G + cta] for j < NV.  Warp sums in the accumulator's
// type, the sum over warps in FP64 in a fixed order.
template <int T, int NV, int NVS, typename AT>
__device__ __forceinline__ void block_cols(AT (&acc)[NV], double* scratch, double* part, int G, int cta,
                                           int j_off = 0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const AT t = col_sum<T>(acc[j]);
        if (lane < T) park(scratch + (warp * T + lane) * NV + j, t);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T * NV; t += kBlock) {
        double sum = 0.0;
        for (int w = 0; w < kWarps; ++w) sum += unpark<AT>(scratch + w * T * NV + t);
        const int c = t / NV, j = t - c * NV;
        part[(size_t)(c * NVS + j_off + j) * G + cta] = sum;
    }
    __syncthreads();
}

// Deterministic grid reduction of value-major partials part[v * G + cta],
// v < nval: a warp takes four values at a time and its lanes read 32
// consecutive CTAs of each (coalesced); every CTA gets bit-identical sums.
__device__ __forceinline__ void grid_sum_vm(const double* part, int G, int nval, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j0 = warp * 4; j0 < nval; j0 += kWarps * 4) {
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (int c0 = 0; c0 < G; c0 += 32 * 4) {
            double v[4][4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = c0 + lane + 32 * u, j = j0 + jj;
                    v[jj][u] = (j < nval && c < G) ? __ldcg(part + (size_t)j * G + c) : 0.0;
                }
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int u = 0; u < 4; ++u) s[jj] += v[jj][u];
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const double t = warp_sum(s[jj]);
            if (lane == 0 && j0 + jj < nval) out[j0 + jj] = t;
        }
    }
    __syncthreads();
}

// A grid barrier that also sums value-major partials part[v * G + cta]
// (v < nval) into out[] (shared) in every CTA: after the barrier CTA c sums
// the values v = c, c + G, ... (one warp each, the CTAs in a fixed order) and
// writes them to res[] (global); a second barrier; then every CTA reads the
// nval sums.  The partials are read once in all, spread over the CTAs, and
// every CTA gets bit-identical sums.  res[] can be reused by the next call: no
// CTA passes that call's first barrier before all have read these sums.
__device__ __forceinline__ bool grid_reduce(const GridSync& g, unsigned long long& epoch, const double* part,
                                            int G, int nval, double* res, double* out) {
    if (!grid_barrier(g, epoch)) return false;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int v = (int)blockIdx.x % G + G * warp; v < nval; v += G * kWarps) {
        const double* pv = part + (size_t)v * G;
        double sum = 0.0;
        for (int c = lane; c < G; c += 32) sum += __ldcg(pv + c);
        sum = warp_sum(sum);
        if (lane == 0) res[v] = sum;
    }
    if (!grid_barrier(g, epoch)) return false;
    for (int t = threadIdx.x; t < nval; t += kBlock) out[t] = __ldcg(res + t);
    __syncthreads();
    return true;
}

// Four consecutive values of a 4x4 block row (16- or 32-byte aligned).
__device__ __forceinline__ void block_row4(const float* p, float (&v)[4]) {
    const float4 t = ld_stream(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void block_row4(const double* p, double (&v)[4]) {
    const double2 a = ld_stream(reinterpret_cast<const double2*>(p));
    const double2 b = ld_stream(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// order-preserving bits of a non-negative double (for atomicMax)
__device__ __forceinline__ unsigned long long key_bits(double v) {
    return (unsigned long long)__double_as_longlong(v);
}

// slots of the blocked apply whose column-block indices are loaded together
// (compensated, 32^3 x 4, 256 right-hand sides: 194.0 us per block iteration
// at T = 32 against 199.0 one at a time; 114.2 against 112.8 at T = 16)
#ifndef SCOCG_BLOCK_SLOT_PRE
#define SCOCG_BLOCK_SLOT_PRE 4
#endif
constexpr int kSlotPre = SCOCG_BLOCK_SLOT_PRE;

template <typename R, int T>
__global__ void __launch_bounds__(kBlock, 2) cocg_block(BlockArgs<R> a) {
    using V = typename Vec<R>::T;
    using W = typename ValT<R>::T;
    using AT = typename Acc<R>::T;
    constexpr int RPW = 32 / T;              // rows a warp covers per step
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ BlockShared<T> s;
    // per slot: z_s, beta_{n-1}, alpha_n in the vector type, converted by the
    // slot's thread when they change rather than by every thread per phase
    __shared__ V s_vz[T], s_vb[T], s_va[T];

    const int G = (int)gridDim.x, cta = (int)blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int sub = lane / T, cl = lane % T;   // this lane's row within the warp step and its slot
    const int64_t rbeg = (int64_t)cta * a.n / G, rend = (int64_t)(cta + 1) * a.n / G;
    const int M = a.nproj, K = a.K;
    const int npairs = T * K;
    const double tol2 = a.tol * a.tol;
    unsigned long long epoch = 0;

    if (tid < T) {
        const bool load = tid < a.nrhs;
        s.rhs[tid] = load ? tid : -1;
        s.state[tid] = load ? kSlotFresh : kSlotEmpty;
        s.n[tid] = 0; s.nsw[tid] = 0; s.siters[tid] = 0; s.pend[tid] = kGoOn;
        s.cnt[tid] = 0; s.bad[tid] = 0; s.sw[tid] = 0;
        s.alpha[tid] = c2(0, 0);
        s_vz[tid] = vzero<V>(); s_vb[tid] = vzero<V>(); s_va[tid] = vzero<V>();
    }
    if (tid == 0) s.next_rhs = a.nrhs < T ? a.nrhs : T;
    __syncthreads();

    bool first = true;
    int nblk = 0;                            // block iterations (every occupied slot advances once)
#ifdef SCOCG_PHASE_TIMERS
    uint64_t t_mark = globaltimer_ns();
#endif
    while (true) {
        SCOCG_MARK(7);
        if (!first) {
            // ---- phase A: q = (z_s - H) r + beta q per running slot; partial r^T q
            {
                AT acc[2] = {};
                const bool run = s.state[cl] == kSlotRun;
                const V zs = s_vz[cl];
                const V bp = s_vb[cl];
                if (a.unit_off) {
                    // block rows: lane group `sub` takes block row B (rows 4B..4B+3);
                    // per column block its lane of slot cl reads the four x entries
                    // once and applies all sixteen block values, so each gathered
                    // x row of T entries serves four rows
                    const int64_t nbr = a.n / 4;
                    const int64_t bbeg = (int64_t)cta * nbr / G, bend = (int64_t)(cta + 1) * nbr / G;
                    for (int64_t b0 = bbeg + warp * RPW; b0 < bend; b0 += kWarps * RPW) {
                        const int64_t B = b0 + sub;
                        if (B >= bend || !run) continue;
                        V rowacc[4] = {vzero<V>(), vzero<V>(), vzero<V>(), vzero<V>()};
                        const int64_t u = B >> 3;
                        const int br = (int)(B & 7);
                        int s0 = a.unit_off[u], s1 = a.unit_off[u + 1];
                        if (!chk(a.dbg, 26, s1, a.nslots + 1) || !chk(a.dbg, 26, s0, s1 + 1)) s0 = s1 = 0;
                        // the column-block indices of kSlotPre slots are loaded
                        // together, so that their gathers need not wait on one
                        // index load each
                        for (int g0 = s0; g0 < s1; g0 += kSlotPre) {
                            int cbs[kSlotPre];
#pragma unroll
                            for (int k = 0; k < kSlotPre; ++k)
                                cbs[k] = g0 + k < s1 ? ld_stream(a.bcol + (size_t)(g0 + k) * 8 + br) : -1;
#pragma unroll
                            for (int k = 0; k < kSlotPre; ++k) {
                                const int cb = cbs[k];
                                if (cb < 0 || !chk(a.dbg, 27, (long long)cb * 4 + 3, a.n)) continue;
                                V xv[4];
#pragma unroll
                                for (int j = 0; j < 4; ++j) xv[j] = a.r[((size_t)cb * 4 + j) * T + cl];
                                const W* hb = a.bval + ((size_t)(g0 + k) * 8 + br) * 16;
#pragma unroll
                                for (int rr = 0; rr < 4; ++rr) {
                                    W hv[4];
                                    block_row4(hb + rr * 4, hv);
#pragma unroll
                                    for (int j = 0; j < 4; ++j) cfma_r(rowacc[rr], hv[j], xv[j]);
                                }
                            }
                        }
#pragma unroll
                        for (int rr = 0; rr < 4; ++rr) {
                            const size_t o = ((size_t)B * 4 + rr) * T + cl;
                            const V ri = a.r[o];
                            const V qn = vcfma(bp, a.q[o], vsub(vcfma(zs, ri, vzero<V>()), rowacc[rr]));
                            a.q[o] = qn;
                            acc_bil(acc[0], acc[1], ri, qn);
                        }
                    }
                }
                for (int64_t i0 = rbeg + warp * RPW; !a.unit_off && i0 < rend; i0 += kWarps * RPW) {
                    const int64_t i = i0 + sub;
                    const bool has = i < rend;
                    int e0 = 0, e1 = 0;
                    if (has) { e0 = a.rowptr[i]; e1 = a.rowptr[i + 1]; }
                    if (!chk(a.dbg, 21, e0, a.nnz + 1) || !chk(a.dbg, 22, e1, a.nnz + 1)) e0 = e1 = 0;
                    V w = vzero<V>();
                    for (int base = e0; __any_sync(kFull, base < e1); base += T) {
                        int cj = 0;
                        W vj = W(0);
                        if (base + cl < e1) { cj = ld_stream(a.col + base + cl); vj = ld_stream(a.val + base + cl); }
                        const int cnt = e1 - base;
#pragma unroll 8
                        for (int j = 0; j < T; ++j) {
                            const int cc = __shfl_sync(kFull, cj, j, T);
                            const W vv = __shfl_sync(kFull, vj, j, T);
                            if (run && j < cnt && chk(a.dbg, 23, cc, a.n)) cfma_r(w, vv, a.r[(size_t)cc * T + cl]);
                        }
                    }
                    if (has && run) {
                        const size_t o = (size_t)i * T + cl;
                        const V ri = a.r[o];
                        const V qn = vcfma(bp, a.q[o], vsub(vcfma(zs, ri, vzero<V>()), w));
                        a.q[o] = qn;
                        acc_bil(acc[0], acc[1], ri, qn);
                    }
                }
                block_cols<T, 2, kNvA>(acc, s.scratch, a.partA, G, cta);
                if (tid < T) {
                    a.partA[(size_t)(tid * kNvA + 2) * G + cta] = (double)s.cnt[tid];
                    a.partA[(size_t)(tid * kNvA + 3) * G + cta] = (double)s.bad[tid];
                }
            }
            SCOCG_MARK(0);
            if (!grid_reduce(a.sync, epoch, a.partA, G, kNvA * T, a.res, s.red)) return;
            SCOCG_MARK(1);

            // ---- decide: alpha per running slot, or finish it
            if (tid < T) {
                const int c = tid;
                int fin = kGoOn;
                if (s.state[c] == kSlotRun) {
                    const double* rd = s.red + kNvA * c;
                    const double2 rq = c2(rd[0], rd[1]);
                    const int active = (int)rd[2];
                    if (s.pend[c] != kGoOn) fin = s.pend[c];
                    else if (rd[3] != 0.0) fin = SCOCG_ERR_BREAKDOWN;
                    else if (active == 0) fin = SCOCG_OK;
                    else if (s.n[c] >= a.max_iter) fin = SCOCG_NOT_CONVERGED;
                    else if (cabs2(s.rho[c]) == 0.0 || cabs2(rq) == 0.0 || !cfinite(rq)) fin = SCOCG_ERR_BREAKDOWN;
                    else {
                        const double2 al = cdiv(s.rho[c], rq);
                        if (!cfinite(al)) fin = SCOCG_ERR_BREAKDOWN;
                        else { s.alpha[c] = al; s_va[c] = Vec<R>::make(al); s.siters[c] += active; }
                    }
                }
                s.fin[c] = fin;
            }
            __syncthreads();
            // outputs of the right-hand sides that finished
            for (int p = cta + G * tid; p < npairs; p += G * kBlock) {
                const int c = p / K, k = p - c * K;
                if (s.fin[c] == kGoOn) continue;
                const int j = s.rhs[c];
                for (int m = 0; m < M; ++m) a.G[((size_t)j * M + m) * K + k] = a.X[(size_t)p * M + m];
                a.out_iters[(size_t)j * K + k] = a.iters[p];
                a.out_resid[(size_t)j * K + k] = a.resid[p];
            }
            if (cta == 0 && tid < T && s.fin[tid] != kGoOn) {
                int* oi = a.out_info + 4 * (size_t)s.rhs[tid];
                oi[0] = s.fin[tid]; oi[1] = s.n[tid]; oi[2] = s.nsw[tid]; oi[3] = s.seed[tid];
            }
            __syncthreads();
            if (tid == 0) {   // refill in slot order: every CTA makes the same assignment
                int live = 0;
                for (int c = 0; c < T; ++c) {
                    if (s.fin[c] != kGoOn) {
                        if (s.next_rhs < a.nrhs) { s.rhs[c] = s.next_rhs++; s.state[c] = kSlotFresh; }
                        else { s.rhs[c] = -1; s.state[c] = kSlotEmpty; }
                    }
                    live |= s.state[c] != kSlotEmpty;
                }
                s.any_live = live;
            }
            __syncthreads();
            if (!s.any_live) break;
            ++nblk;
            SCOCG_MARK(6);
        }
        first = false;

        // ---- phase B: r -= alpha q (running), r = b and q = 0 (refilled)
        {
            AT acc[3] = {};
            double nb[1] = {0.0};
            const int st = s.state[cl];
            const V al = s_va[cl];
            const double2* bj = st == kSlotFresh ? a.b + (size_t)s.rhs[cl] * a.n : nullptr;
            constexpr int64_t kStep = (int64_t)kWarps * RPW;
            if (st == kSlotRun) {
                // one row ahead: the next row's r and q are in flight while this
                // row is updated and stored (same rows, same order per lane)
                int64_t i = rbeg + warp * RPW + sub;
                V r0 = vzero<V>(), q0 = vzero<V>();
                if (i < rend) { r0 = a.r[(size_t)i * T + cl]; q0 = a.q[(size_t)i * T + cl]; }
                for (; i < rend; i += kStep) {
                    const int64_t inx = i + kStep;
                    V r1 = vzero<V>(), q1 = vzero<V>();
                    if (inx < rend) { r1 = a.r[(size_t)inx * T + cl]; q1 = a.q[(size_t)inx * T + cl]; }
                    const V rn = r_update(r0, al, q0);
                    a.r[(size_t)i * T + cl] = rn;
                    acc_rr(acc[0], acc[1], acc[2], rn);
                    r0 = r1; q0 = q1;
                }
            }
            for (int64_t i0 = rbeg + warp * RPW; st == kSlotFresh && i0 < rend; i0 += kStep) {
                const int64_t i = i0 + sub;
                if (i >= rend) continue;
                const size_t o = (size_t)i * T + cl;
                const double2 bi = bj[i];
                const V rn = Vec<R>::make(bi);
                a.q[o] = vzero<V>();
                nb[0] = fma(bi.x, bi.x, fma(bi.y, bi.y, nb[0]));
                a.r[o] = rn;
                acc_rr(acc[0], acc[1], acc[2], rn);
            }
            block_cols<T, 3, kNvB>(acc, s.scratch, a.partB, G, cta);
            block_cols<T, 1, kNvB>(nb, s.scratch, a.partB, G, cta, 3);
        }
        SCOCG_MARK(2);
        if (!grid_reduce(a.sync, epoch, a.partB, G, kNvB * T, a.res, s.red)) return;
        SCOCG_MARK(3);
        if (tid < T) {
            const int c = tid;
            const double* rd = s.red + kNvB * c;
            if (s.state[c] == kSlotRun) {
                s.rho_new[c] = c2(rd[0], rd[1]);
                s.t2[c] = cdiv(cmul(s.alpha[c], s.beta_prev[c]), s.alpha_prev[c]);
                const double rn_b = sqrt(rd[2]) / s.bnorm[c];
                s.rn_b2[c] = rn_b * rn_b;
            } else if (s.state[c] == kSlotFresh) {
                s.rho[c] = c2(rd[0], rd[1]);
                s.bnorm[c] = sqrt(rd[3]);
                s.alpha_prev[c] = c2(1, 0);
                s.beta_prev[c] = c2(0, 0);
                s.seed[c] = a.seed0;
                s.zs[c] = a.z[a.seed0];
                s_vz[c] = Vec<R>::make(s.zs[c]);
                s_vb[c] = vzero<V>();
                s.n[c] = 0; s.nsw[c] = 0; s.pend[c] = kGoOn;
            }
            s.cnt[c] = 0; s.bad[c] = 0;
        }
        // unit projections c_m^T r of the new residual (or of r_0 = b)
        for (int t = tid; t < T * M; t += kBlock) {
            const int c = t / M, m = t - c * M;
            if (s.state[c] == kSlotEmpty) continue;
            const int64_t idx = a.cidx[(size_t)s.rhs[c] * M + m];
            s.cr_next[t] = chk(a.dbg, 24, idx, a.n) ? Vec<R>::wide(__ldcg(a.r + (size_t)idx * T + c)) : c2(0, 0);
        }
        __syncthreads();
        SCOCG_MARK(5);

        // ---- phase C: per (slot, shift) pair
        for (int p = cta + G * tid; p < npairs; p += G * kBlock) {
            const int c = p / K, k = p - c * K;
            const int st = s.state[c];
            if (st == kSlotEmpty) continue;
            if (st == kSlotFresh) {
                a.pi_prev[p] = c2(1, 0); a.pi_cur[p] = c2(1, 0); a.inv_cur[p] = c2(1, 0);
                a.sigma[p] = csub(a.z[k], a.z[a.seed0]);
                a.alpha_k[p] = c2(0, 0);
                for (int m = 0; m < M; ++m) { a.P[(size_t)p * M + m] = c2(0, 0); a.X[(size_t)p * M + m] = c2(0, 0); }
                const bool zero = s.bnorm[c] == 0.0;   // b = 0: x = 0 solves every shift
                a.frozen[p] = zero; a.iters[p] = 0; a.resid[p] = zero ? 0.0 : 1.0;
                if (!zero) atomicAdd(&s.cnt[c], 1);
                continue;
            }
            if (a.frozen[p]) continue;
            const double2 al = s.alpha[c];
            const double2 pp = a.pi_prev[p], pc = a.pi_cur[p], ic = a.inv_cur[p];
            const double2 ratio = cmul(pp, ic);
            const double2 beta_k = cmul(cmul(ratio, ratio), s.beta_prev[c]);
            const double2 pn = cadd(cmul(cadd(c2(1, 0), cmul(al, a.sigma[p])), pc), cmul(s.t2[c], csub(pc, pp)));
            const double2 in = crecip(pn);
            if (cabs2(pn) == 0.0 || !cfinite(pn) || !cfinite(in)) {
                atomicOr(&s.bad[c], 1);
                continue;
            }
            const double2 ak = cmul(cmul(pc, in), al);
            for (int m = 0; m < M; ++m) {
                const size_t o = (size_t)p * M + m;
                const double2 Pm = cadd(cmul(s.cr_cur[c * M + m], ic), cmul(beta_k, a.P[o]));
                a.P[o] = Pm;
                a.X[o] = cadd(a.X[o], cmul(ak, Pm));
            }
            a.alpha_k[p] = ak;
            a.pi_prev[p] = pc;
            a.pi_cur[p] = pn;
            a.inv_cur[p] = in;
            const double res2 = s.rn_b2[c] * cabs2(in);
            a.resid[p] = res2;
            a.iters[p] = s.n[c] + 1;
            if (a.tol > 0.0 && res2 <= tol2) a.frozen[p] = 1;
            else atomicAdd(&s.cnt[c], 1);
        }
        __syncthreads();
        if (tid < T) {
            const int c = tid;
            s.sw[c] = 0;
            if (s.state[c] == kSlotRun) {
                s.beta_prev[c] = cdiv(s.rho_new[c], s.rho[c]);
                s_vb[c] = Vec<R>::make(s.beta_prev[c]);
                s.alpha_prev[c] = s.alpha[c];
                s.rho[c] = s.rho_new[c];
                s.n[c] += 1;
                // the seed (pi = 1) has converged while shifts remain: switch
                s.sw[c] = a.tol > 0.0 && s.rn_b2[c] <= tol2;
            } else if (s.state[c] == kSlotFresh) {
                s.state[c] = kSlotRun;
            }
            s.key[c] = 0ull; s.arg[c] = INT_MAX;
        }
        for (int t = tid; t < T * M; t += kBlock) s.cr_cur[t] = s.cr_next[t];
        SCOCG_MARK(4);

        // ---- seed switching (Sec. III.C) for the slots whose seed converged
        if (__syncthreads_or(tid < T && s.sw[tid])) {
            // local candidate per slot: the unconverged shift with the smallest
            // |pi| (largest residual), lowest index on ties
            for (int p = cta + G * tid; p < npairs; p += G * kBlock) {
                const int c = p / K;
                if (s.sw[c] && !a.frozen[p]) atomicMax(&s.key[c], key_bits(cabs2(a.inv_cur[p])));
            }
            __syncthreads();
            for (int p = cta + G * tid; p < npairs; p += G * kBlock) {
                const int c = p / K, k = p - c * K;
                if (s.sw[c] && !a.frozen[p] && key_bits(cabs2(a.inv_cur[p])) == s.key[c]) atomicMin(&s.arg[c], k);
            }
            __syncthreads();
            for (int p = cta + G * tid; p < npairs; p += G * kBlock) {
                const int c = p / K, k = p - c * K;
                if (!s.sw[c] || a.frozen[p] || k != s.arg[c]) continue;
                // the candidate's recurrence values travel with it
                double* pc = a.partC + (size_t)(c * kNvC) * G + cta;
                const double2 pp = a.pi_prev[p], pq = a.pi_cur[p], ak = a.alpha_k[p];
                pc[4 * G] = pp.x; pc[5 * G] = pp.y; pc[6 * G] = pq.x; pc[7 * G] = pq.y;
                pc[8 * G] = ak.x; pc[9 * G] = ak.y;
            }
            if (tid < T && s.sw[tid]) {
                double* pc = a.partC + (size_t)(tid * kNvC) * G + cta;
                const bool any = s.arg[tid] != INT_MAX;
                pc[0] = (double)s.cnt[tid];
                pc[G] = any ? __longlong_as_double((long long)s.key[tid]) : -1.0;
                pc[2 * G] = any ? (double)s.arg[tid] : (double)INT_MAX;
                pc[3 * G] = (double)s.bad[tid];
            }
            if (!grid_barrier(a.sync, epoch)) return;
            if (tid < T) {
                const int c = tid;
                int go = 0;
                if (s.sw[c]) {
                    double tot = 0.0, bad = 0.0, gbest = -1.0;
                    int garg = INT_MAX, gc = -1;
                    for (int g = 0; g < G; ++g) {
                        const double* pc = a.partC + (size_t)(c * kNvC) * G + g;
                        tot += __ldcg(pc);
                        bad += __ldcg(pc + 3 * G);
                        const double kb = __ldcg(pc + G);
                        const int ka = (int)__ldcg(pc + 2 * G);
                        if (kb > gbest || (kb == gbest && ka < garg)) { gbest = kb; garg = ka; gc = g; }
                    }
                    if (tot == 0.0 || bad != 0.0) {
                        go = 0;   // all converged, or a failure the next decision reports
                    } else if (!a.allow_switch || gc < 0 || !chk(a.dbg, 25, garg, K)) {
                        s.pend[c] = SCOCG_ERR_BREAKDOWN;
                    } else {
                        const double* pc = a.partC + (size_t)(c * kNvC) * G + gc;
                        const double2 pin = c2(__ldcg(pc + 4 * G), __ldcg(pc + 5 * G));    // pi^{s'}_n
                        const double2 pin1 = c2(__ldcg(pc + 6 * G), __ldcg(pc + 7 * G));   // pi^{s'}_{n+1}
                        const double2 as2 = c2(__ldcg(pc + 8 * G), __ldcg(pc + 9 * G));    // alpha^{s'}_n
                        // r' = r_{n+1} / pi'_{n+1};  q' = (r_n / pi'_n - r_{n+1} / pi'_{n+1}) / alpha'_n
                        const double2 inv1 = cdiv(c2(1, 0), pin1);
                        s.sw_inv1[c] = inv1;
                        s.sw_ca[c] = cdiv(csub(cdiv(c2(1, 0), pin), inv1), as2);
                        s.sw_cb[c] = cdiv(cdiv(s.alpha_prev[c], pin), as2);
                        s.sw_pin[c] = pin; s.sw_pin1[c] = pin1; s.sw_alpha[c] = as2;
                        s.s2[c] = garg;
                        go = 1;
                    }
                }
                s.sw[c] = go;
            }
            if (__syncthreads_or(tid < T && s.sw[tid])) {
                {
                    const bool mine = s.sw[cl] != 0;
                    const V v_inv1 = Vec<R>::make(s.sw_inv1[cl]);
                    const V v_ca = Vec<R>::make(s.sw_ca[cl]), v_cb = Vec<R>::make(s.sw_cb[cl]);
                    for (int64_t i0 = rbeg + warp * RPW; i0 < rend && mine; i0 += kWarps * RPW) {
                        const int64_t i = i0 + sub;
                        if (i >= rend) continue;
                        const size_t o = (size_t)i * T + cl;
                        const V ri = a.r[o], qi = a.q[o];
                        a.q[o] = vcfma(v_cb, qi, vcfma(v_ca, ri, vzero<V>()));
                        a.r[o] = vcfma(v_inv1, ri, vzero<V>());
                    }
                }
                for (int p = cta + G * tid; p < npairs; p += G * kBlock) {
                    const int c = p / K, k = p - c * K;
                    if (!s.sw[c]) continue;
                    if (k == s.s2[c]) {
                        a.pi_prev[p] = c2(1, 0); a.pi_cur[p] = c2(1, 0); a.inv_cur[p] = c2(1, 0);
                    } else {
                        a.pi_prev[p] = cdiv(a.pi_prev[p], s.sw_pin[c]);
                        a.pi_cur[p] = cdiv(a.pi_cur[p], s.sw_pin1[c]);
                        a.inv_cur[p] = cmul(a.inv_cur[p], s.sw_pin1[c]);
                    }
                    a.sigma[p] = csub(a.z[k], a.z[s.s2[c]]);
                }
                for (int t = tid; t < T * M; t += kBlock) {
                    const int c = t / M;
                    if (s.sw[c]) s.cr_cur[t] = cmul(s.cr_cur[t], s.sw_inv1[c]);
                }
                __syncthreads();
                if (tid < T && s.sw[tid]) {
                    const int c = tid;
                    const double2 ratio = cdiv(s.sw_pin[c], s.sw_pin1[c]);
                    s.rho[c] = cdiv(s.rho[c], cmul(s.sw_pin1[c], s.sw_pin1[c]));
                    s.beta_prev[c] = cmul(cmul(ratio, ratio), s.beta_prev[c]);
                    s.alpha_prev[c] = s.sw_alpha[c];
                    s.seed[c] = s.s2[c];
                    s.zs[c] = a.z[s.s2[c]];
                    s_vz[c] = Vec<R>::make(s.zs[c]);
                    s_vb[c] = Vec<R>::make(s.beta_prev[c]);
                    s.nsw[c] += 1;
                }
                if (!grid_barrier(a.sync, epoch)) return;
            }
        }
    }

    if (cta == 0 && tid == 0) {
        long long si = 0;
        for (int c = 0; c < T; ++c) si += s.siters[c];
        a.stats->shift_iters = si;
        a.stats->iters = nblk;
        a.stats->status = SCOCG_OK;
    }
}

}  // namespace scocg
