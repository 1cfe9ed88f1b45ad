// Body of the persistent single-right-hand-side shifted-COCG kernel.  See
// solver.cuh for the algorithm; this file holds the phases.
#pragma once
#include <type_traits>

#include "solver.cuh"

namespace scocg {

// A warp sum parked in a double-sized scratch slot in its own type, so that
// only the final sum over warps (NV threads of warp 0) uses the FP64 pipe:
// on this GPU an FP64 instruction issued by every warp of an SM holds the
// FP64 pipe for hundreds of cycles.
__device__ __forceinline__ void park(double* slot, double v) { *slot = v; }
__device__ __forceinline__ void park(double* slot, float v) { *reinterpret_cast<float*>(slot) = v; }
__device__ __forceinline__ void park(double* slot, dfs v) { *reinterpret_cast<dfs*>(slot) = v; }
template <typename T> __device__ __forceinline__ double unpark(const double* slot);
template <> __device__ __forceinline__ double unpark<double>(const double* slot) { return *slot; }
template <> __device__ __forceinline__ double unpark<float>(const double* slot) {
    return (double)*reinterpret_cast<const float*>(slot);
}
template <> __device__ __forceinline__ double unpark<dfs>(const double* slot) {
    return to_double(*reinterpret_cast<const dfs*>(slot));
}

// CTA sum of per-thread values: the warp-level part in the values' own type
// (FP32 for complex64 vectors), the sum over warps in FP64.
template <int NV, typename T>
__device__ __forceinline__ void block_sum_n(T (&v)[NV], double* scratch, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if constexpr (std::is_same<T, double>::value) {
        // FP64 values: every thread parks its values (scratch holds NV *
        // kBlock doubles) and NV warps sum them, instead of NV five-step FP64
        // warp sums in all kWarps warps (an FP64 instruction of a whole warp
        // occupies the FP64 pipe ~16 cycles)
        static_assert(NV <= kScratchNV, "scratch too small");
#pragma unroll
        for (int j = 0; j < NV; ++j) scratch[j * kBlock + threadIdx.x] = v[j];
        __syncthreads();
        if (warp < NV) {
            double acc = 0.0;
            for (int t = lane; t < kBlock; t += 32) acc += scratch[warp * kBlock + t];
            acc = warp_sum(acc);
            if (lane == 0) out[warp] = acc;
        }
        __syncthreads();
    } else {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const T t = warp_sum(v[j]);
            if (lane == 0) park(scratch + warp * NV + j, t);
        }
        __syncthreads();
        if (threadIdx.x < NV) {
            double s = 0.0;
            for (int w = 0; w < kWarps; ++w) s += unpark<T>(scratch + w * NV + threadIdx.x);
            out[threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// per-thread accumulation of u^T v (bilinear) in the vector precision
__device__ __forceinline__ void acc_bil(double& re, double& im, double2 u, double2 v) {
    re = fma(u.x, v.x, fma(-u.y, v.y, re)); im = fma(u.x, v.y, fma(u.y, v.x, im));
}
__device__ __forceinline__ void acc_bil(float& re, float& im, float2 u, float2 v) {
    re = fmaf(u.x, v.x, fmaf(-u.y, v.y, re)); im = fmaf(u.x, v.y, fmaf(u.y, v.x, im));
}
__device__ __forceinline__ void acc_nrm(double& s, double2 u) { s = fma(u.x, u.x, fma(u.y, u.y, s)); }
__device__ __forceinline__ void acc_nrm(float& s, float2 u) { s = fmaf(u.x, u.x, fmaf(u.y, u.y, s)); }
// compensated: products exact to DF, sums with TwoSum; the real and
// imaginary parts as one packed pair, (re, im) += (u.re, u.re) (v.re, v.im)
// + (-u.im, u.im) (v.im, v.re)
__device__ __forceinline__ void acc_bil(dfs& re, dfs& im, float4 u, float4 v) {
    float2 h = make_float2(re.hi, im.hi), l = make_float2(re.lo, im.lo);
    pk_acc_prod(h, l, make_float2(u.x, u.x), make_float2(u.z, u.z), hi2(v), lo2(v));
    pk_acc_prod(h, l, make_float2(-u.y, u.y), make_float2(-u.w, u.w), make_float2(v.y, v.x), make_float2(v.w, v.z));
    re = dfs{h.x, l.x};
    im = dfs{h.y, l.y};
}
__device__ __forceinline__ void acc_nrm(dfs& s, float4 u) {
    df_acc_prod(s, cre(u), cre(u));
    df_acc_prod(s, cim(u), cim(u));
}

// Per-thread accumulation of rho = r^T r (re, im) and ||r||^2.
template <typename AT, typename V>
__device__ __forceinline__ void acc_rr(AT& re, AT& im, AT& nrm, V ri) {
    acc_bil(re, im, ri, ri);
    acc_nrm(nrm, ri);
}
// Compensated vectors: rho = sum (x^2 - y^2) + 2i sum x y from three
// pair-exact products (the doubling is exact), and ||r||^2 from the high
// parts in FP32: it only feeds the convergence test, where a relative
// accuracy of 1e-7 is ample.
template <>
__device__ __forceinline__ void acc_rr<dfs, float4>(dfs& re, dfs& im, dfs& nrm, float4 ri) {
    // (re, im) += (x, x) (x, 2y) + (-y, 0) (y, 0), packed
    float2 h = make_float2(re.hi, im.hi), l = make_float2(re.lo, im.lo);
    pk_acc_prod(h, l, make_float2(ri.x, ri.x), make_float2(ri.z, ri.z), make_float2(ri.x, 2.f * ri.y),
                make_float2(ri.z, 2.f * ri.w));
    pk_acc_prod(h, l, make_float2(-ri.y, 0.f), make_float2(-ri.w, 0.f), make_float2(ri.y, 0.f),
                make_float2(ri.w, 0.f));
    re = dfs{h.x, l.x};
    im = dfs{h.y, l.y};
    nrm.hi = fmaf(ri.x, ri.x, fmaf(ri.y, ri.y, nrm.hi));
}

// Per-thread accumulation of the r partials: rho = r^T r, ||r||^2, c_0^T r.
template <typename R>
__device__ __forceinline__ void acc_r(typename Acc<R>::T (&acc)[5], typename Vec<R>::T ri,
                                     const typename Vec<R>::T* c0) {
    acc_rr(acc[0], acc[1], acc[2], ri);
    if (c0) acc_bil(acc[3], acc[4], *c0, ri);
}

// r_{n+1} = r_n - alpha_n q_n (one fused multiply-add for compensated vectors)
template <typename V>
__device__ __forceinline__ V r_update(V r, V al, V q) { return vsub(r, vcfma(al, q, vzero<V>())); }
template <>
__device__ __forceinline__ float4 r_update<float4>(float4 r, float4 al, float4 q) {
    return vcfma(make_float4(-al.x, -al.y, -al.z, -al.w), q, r);
}

// CTA sum of the accumulated partials into values 0..4 of this CTA's column
// of the value-major partials (value j at part[j * G]); the extra dense
// projections m >= 1 are summed in separate passes over r into values 3 + 2m.
template <typename R>
__device__ __forceinline__ void finish_r_partials(const SolveArgs<R>& a, const typename Acc<R>::T (&acc)[5],
                                                  int64_t rbeg, int64_t rend, SeedScalars& s, double* s_part,
                                                  double* part, int G) {
    using AT = typename Acc<R>::T;
    const int tid = threadIdx.x;
    AT v[5] = {acc[0], acc[1], acc[2], acc[3], acc[4]};
    block_sum_n<5>(v, s.scratch, s_part);
    if (tid < 5) part[(size_t)tid * G] = s_part[tid];
    for (int m = 1; m < a.nproj && a.cvec; ++m) {
        AT w2[2] = {};
        for (int64_t i = rbeg + tid; i < rend; i += kBlock) acc_bil(w2[0], w2[1], a.cvec[(size_t)m * a.n + i], a.r[i]);
        block_sum_n<2>(w2, s.scratch, s_part);
        if (tid < 2) part[(size_t)(3 + 2 * m + tid) * G] = s_part[tid];
    }
}

template <typename R>
__device__ __forceinline__ void r_partials(const SolveArgs<R>& a, int64_t rbeg, int64_t rend,
                                           SeedScalars& s, double* s_part, double* part, int G) {
    typename Acc<R>::T acc[5] = {};
    for (int64_t i = rbeg + threadIdx.x; i < rend; i += kBlock)
        acc_r<R>(acc, a.r[i], a.cvec ? a.cvec + i : nullptr);
    finish_r_partials(a, acc, rbeg, rend, s, s_part, part, G);
}

#ifdef SCOCG_CHECKED
#define SCOCG_TRACE(ph)                                                    \
    do {                                                                   \
        if (threadIdx.x == 0 && a.trace) {                                 \
            volatile int* t_ = a.trace + 2 * cta;                          \
            t_[0] = s.n; t_[1] = (ph);                                     \
            __threadfence_system();                                        \
        }                                                                  \
    } while (0)
#else
#define SCOCG_TRACE(ph) do { } while (0)
#endif

// Optional per-phase wall-time accounting (-DSCOCG_PHASE_TIMERS): thread 0 of
// each CTA adds the time spent since the previous mark to slot `k` of its row in
// a.phase_ns ([grid][8] nanoseconds).
#ifdef SCOCG_PHASE_TIMERS
#define SCOCG_MARK(k)                                                      \
    do {                                                                   \
        if (threadIdx.x == 0 && a.phase_ns) {                              \
            const uint64_t t_ = globaltimer_ns();                          \
            a.phase_ns[8 * cta + (k)] += t_ - t_mark;                      \
            t_mark = t_;                                                   \
        }                                                                  \
    } while (0)
#else
#define SCOCG_MARK(k) do { } while (0)
#endif

// The inputs of one phase C (the per-shift update of seed iteration n): the
// seed scalars alpha_n, beta_{n-1}, alpha_n beta_{n-1} / alpha_{n-1},
// (||r_{n+1}|| / ||b||)^2 and c_m^T r_n.  Phase C can run one iteration late,
// inside the next phase A, from this copy.
struct ShiftInputs {
    double2 alpha, beta_prev, t2;
    double rn_b2;
    int n;
    double2 cr[kMaxProj];
};

// Phase C for shift k: the pi three-term recurrence, the projected p^k and
// x^k, the residual estimate and freezing.  Sets bad for a zero or non-finite
// pi, active when the shift stays unconverged.
template <typename R>
__device__ __forceinline__ void shift_update(const SolveArgs<R>& a, int k, const ShiftInputs& c, int M,
                                             double tol2, int& active, int& bad) {
    const double2 pp = a.S.pi_prev[k], pc = a.S.pi_cur[k], ic = a.S.inv_cur[k];
    const double2 ratio = cmul(pp, ic);                        // pi_{n-1} / pi_n
    const double2 beta_k = cmul(cmul(ratio, ratio), c.beta_prev);
    const double2 pn = cadd(cmul(cadd(c2(1, 0), cmul(c.alpha, a.S.sigma[k])), pc), cmul(c.t2, csub(pc, pp)));
    const double2 in = crecip(pn);
    if (cabs2(pn) == 0.0 || !cfinite(pn) || !cfinite(in)) {
        bad = 1;
        return;
    }
    const double2 ak = cmul(cmul(pc, in), c.alpha);            // alpha^k_n
    for (int m = 0; m < M; ++m) {
        const size_t o = (size_t)k * M + m;
        const double2 P = cadd(cmul(c.cr[m], ic), cmul(beta_k, a.S.P[o]));
        a.S.P[o] = P;
        a.S.X[o] = cadd(a.S.X[o], cmul(ak, P));
    }
    a.S.alpha_k[k] = ak;
    a.S.pi_prev[k] = pc;
    a.S.pi_cur[k] = pn;
    a.S.inv_cur[k] = in;
    const double res2 = c.rn_b2 * cabs2(in);
    a.S.resid[k] = res2;
    a.S.iters[k] = c.n + 1;
    if (a.tol > 0.0 && res2 <= tol2) a.S.frozen[k] = 1;
    else active = 1;
}

// Applies whose phase A runs in two passes (they declare kTwoPass and
// provide pass1 / pass2, see ApplyHubbard).
template <class A, class = void>
struct HasTwoPass : std::false_type {};
template <class A>
struct HasTwoPass<A, std::void_t<decltype(A::kTwoPass)>> : std::integral_constant<bool, A::kTwoPass> {};

// Decision word of the per-iteration checks: kGoOn continues, any other value
// ends the solve with that status (SCOCG_OK is 0, so 0 cannot mean "go on").
constexpr int kGoOn = 0x7fffffff;

// The first phase A of a solve continued from a ResumeState: the stopped
// apply's r^T q partial again, from the stored r_n and q_n over the same rows
// in the same order (so the continued solve matches an uninterrupted one bit
// for bit), and the shift count as its deferred phase C left it.
template <typename R, class Apply>
__device__ __forceinline__ void resume_partials(const SolveArgs<R>& a, const Apply& ap, int G, int cta, int64_t ubeg,
                                             int64_t u_end, int64_t u_step, bool active, SeedScalars& s,
                                             double* s_part) {
    using AT = typename Acc<R>::T;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool rot = a.rstate->rotated != 0;
    const int wi = rot ? (warp + kWarps - 1) % kWarps : warp;
    const int64_t first = Apply::kMap == kMapStrided ? (int64_t)cta + (int64_t)G * wi : ubeg + wi;
    AT rq[2] = {};
    for (int64_t u = first; u < u_end; u += u_step) {
        int64_t row;
        if (ap.row_of(u, lane, row)) acc_bil(rq[0], rq[1], a.r[row], a.q[row]);
    }
    const int act = __syncthreads_count(active);
    block_sum_n<2>(rq, s.scratch, s_part);
    if (tid == 0) {
        double* pa = a.partA + cta;
        pa[0] = s_part[0]; pa[G] = s_part[1];
        pa[2 * G] = (double)act;
        pa[3 * G] = 0.0;
    }
    __syncthreads();
}

// Thread 0 of CTA 0 at the end of a solve: the state a later launch continues
// from when the solve stopped at max_iter (right after the apply of iteration
// n).  Out of line, so that the solve loop's code is the same with or without it.
static __device__ __noinline__ void save_resume_state(ResumeState* rs, const SeedScalars& s, int status, int M,
                                               bool rotated) {
    rs->valid = status == SCOCG_NOT_CONVERGED;
    rs->n = s.n; rs->seed = s.seed; rs->n_switch = s.n_switch; rs->n_replace = s.n_replace;
    rs->replace_on = s.replace_on;
    rs->rotated = rotated;
    rs->alpha_prev = s.alpha_prev; rs->beta_prev = s.beta_prev; rs->rho = s.rho; rs->rho_prev = s.rho_prev;
    rs->zs = s.zs; rs->rnorm = s.rnorm; rs->bnorm = s.bnorm;
    for (int m = 0; m < M; ++m) rs->cr_cur[m] = s.cr_cur[m];
}

// The whole solve of one system, run by its G co-resident CTAs (this one is
// number cta among them).
// kResume: the instantiation that continues a stopped solve (a.resume = 1):
// its init takes the stored state and its first phase A only forms the
// stopped apply's partials again.
template <typename R, class Apply, bool kResume = false>
__device__ __forceinline__ void cocg_body(const SolveArgs<R>& a, const Apply& ap, const int G, const int cta) {
    using V = typename Vec<R>::T;
    using AT = typename Acc<R>::T;
    constexpr bool kMixed = std::is_same<R, float>::value;   // complex64 vectors
    constexpr bool kFull = std::is_same<R, double>::value;   // full-vector mode compiled (FP64 only)
    __shared__ SeedScalars s;
    __shared__ double s_part[8];
    __shared__ int s_flag[5];
    __shared__ double s_min[kWarps];
    __shared__ int s_arg[kWarps];
    __shared__ ShiftInputs s_c;          // inputs of a deferred phase C
    // z_s, beta_{n-1}, alpha_n in the vector type, converted once by thread 0
    // whenever they change (every thread converting them would queue all
    // warps on the FP64 pipe at each phase start)
    __shared__ V s_vs[3];
    SCOCG_DYN_SHARED(double2, s_full);   // full-vector mode: per-shift scalars of the iteration

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    // phase A visits units in the apply's order (kMap); the row-wise phases
    // use a contiguous row range per CTA.
    const int64_t ubeg = (int64_t)cta * a.nunits / G, uend = (int64_t)(cta + 1) * a.nunits / G;
    constexpr bool kWhole = Apply::kMap != kMapContiguous;   // every CTA visits the whole unit range
    const int64_t u_first = Apply::kMap == kMapStrided ? (int64_t)cta + (int64_t)G * warp : ubeg + warp;
    const int64_t u_step = kWhole ? (int64_t)G * kWarps : kWarps;
    const int64_t u_end = kWhole ? a.nunits : uend;
    const int64_t rbeg = (int64_t)cta * a.n / G, rend = (int64_t)(cta + 1) * a.n / G;
    const int M = a.nproj;
    const bool dense_proj = a.cvec != nullptr;
    const int nred = dense_proj ? 3 + 2 * M : 3;
    double* myB = a.partB + cta;              // value-major partials: value j at myB[j * G]
    unsigned long long epoch = 0;
    const double tol2 = a.tol * a.tol;
    const int k_own = cta + tid * G;          // the shift this thread owns (if < K)
    const bool owns = k_own < a.K;
    // Phase C may be deferred into the next phase A when every shift owner of
    // every CTA is in warp 0 (K <= 32 G) and no per-shift vectors are formed:
    // warp 0 then updates the shifts while the other warps apply H.  Seed
    // switching needs the shifts of the same iteration, so an iteration whose
    // seed has converged runs phase C in place.
    bool defer_ok = a.K <= 32 * G;
    if constexpr (kFull) defer_ok = defer_ok && a.Xf == nullptr;
    bool pending = false;                     // a deferred phase C waits for the next phase A

    int status = SCOCG_NOT_CONVERGED;
    bool done = false;
#ifdef SCOCG_PHASE_TIMERS
    uint64_t t_mark = globaltimer_ns();
#endif

    // ------------------------------------------------------------ init: r_0 = b, q_{-1} = 0
    // (or, continuing a solve stopped at max_iter, the stored state)
    if constexpr (kResume) {
        if (tid == 0) {
            const ResumeState& rs = *a.rstate;
            s.rho = rs.rho; s.rho_prev = rs.rho_prev;
            s.alpha_prev = rs.alpha_prev; s.beta_prev = rs.beta_prev;
            s.bnorm = rs.bnorm; s.rnorm = rs.rnorm;
            s.seed = rs.seed; s.zs = rs.zs;
            s_vs[0] = Vec<R>::make(s.zs);
            s_vs[1] = Vec<R>::make(s.beta_prev);
            s.n = rs.n;
            s.active = a.K;
            s.replace_on = rs.replace_on; s.n_switch = rs.n_switch; s.n_replace = rs.n_replace;
            s.shift_iters = 0;
        }
        if (tid < M) s.cr_cur[tid] = a.rstate->cr_cur[tid];
        // s_flag[4] (seed converged) decides whether the next apply takes a
        // deferred shift update and visits its units rotated: restored so
        // that a stop right after this pass records the stopped one's order
        if (tid < 5) s_flag[tid] = tid == 4 ? (a.rstate->rotated ? 0 : 1) : 0;
        __syncthreads();
        resume_partials(a, ap, G, cta, ubeg, u_end, u_step, owns && !a.S.frozen[k_own], s, s_part);
    } else {
        double nb = 0.0;
        for (int64_t i = rbeg + tid; i < rend; i += kBlock) {
            const double2 bi = a.b[i];
            a.r[i] = Vec<R>::make(bi);
            a.q[i] = vzero<V>();
            if constexpr (kMixed) {
                a.p_seed[i] = vzero<V>(); a.x_hi[i] = vzero<V>(); a.x_lo[i] = vzero<V>();
            }
            if constexpr (kFull)
                if (a.Xf)
                    for (int k = 0; k < a.K; ++k) { a.Xf[(size_t)k * a.n + i] = c2(0, 0); a.Pf[(size_t)k * a.n + i] = c2(0, 0); }
            nb = fma(bi.x, bi.x, fma(bi.y, bi.y, nb));
        }
        double v1[1] = {nb};
        block_sum_n<1>(v1, s.scratch, s_part);
        if (tid == 0) a.partC[(size_t)cta * kPartC] = s_part[0];
        __syncthreads();
        r_partials(a, rbeg, rend, s, s_part, myB, G);
        if (owns) {
            const int k = k_own;
            a.S.pi_prev[k] = c2(1, 0); a.S.pi_cur[k] = c2(1, 0); a.S.inv_cur[k] = c2(1, 0);
            a.S.sigma[k] = csub(a.z[k], a.z[a.seed]);
            a.S.alpha_k[k] = c2(0, 0);
            for (int m = 0; m < M; ++m) { a.S.P[(size_t)k * M + m] = c2(0, 0); a.S.X[(size_t)k * M + m] = c2(0, 0); }
            a.S.frozen[k] = 0; a.S.iters[k] = 0; a.S.resid[k] = 1.0;
        }
        if (tid < 5) s_flag[tid] = 0;
        if (!grid_barrier(a.sync, epoch)) return;
        grid_sum_vm1(a.partB, nred, s.red, G);
        grid_sum(a.partC, kPartC, 1, s.red + nred, G);
        if (tid == 0) {
            s.rho = c2(s.red[0], s.red[1]);
            s.bnorm = sqrt(s.red[nred]);
            s.rnorm = s.bnorm;
            s.alpha_prev = c2(1, 0);
            s.beta_prev = c2(0, 0);
            s.seed = a.seed;
            s.zs = a.z[a.seed];
            s_vs[0] = Vec<R>::make(s.zs);
            s_vs[1] = Vec<R>::make(s.beta_prev);
            s.n = 0;
            s.active = a.K;
            s.replace_on = kMixed && a.replace_every > 0;
            s.n_switch = 0; s.n_replace = 0; s.shift_iters = 0;
        }
        if (tid < M) {
            s.cr_cur[tid] = dense_proj ? c2(s.red[3 + 2 * tid], s.red[4 + 2 * tid])
                                       : (chk(a.dbg, 12, a.cidx[tid], a.n) ? Vec<R>::wide(__ldcg(a.r + a.cidx[tid])) : c2(0, 0));
        }
        __syncthreads();
        if (s.bnorm == 0.0) {                 // b = 0: x = 0 solves every shift
            if (owns) { a.S.frozen[k_own] = 1; a.S.resid[k_own] = 0.0; }
            status = SCOCG_OK;
            done = true;
        }
    }

    // ------------------------------------------------------------ iterations
    bool skip_a = kResume;                    // the continued solve's first phase A ran before it stopped
    while (!done) {
        SCOCG_TRACE(1);
        SCOCG_MARK(7);
        // ---- phase A: q_n = (z_s - H) r_n + beta_{n-1} q_{n-1}; partial r_n^T q_n
        // (with a deferred phase C of iteration n-1 in warp 0)
        if (!skip_a) {
            const V zs = s_vs[0];
            const V bp = s_vs[1];
            AT rq[2] = {};
            const bool c_here = pending;           // uniform over the grid
            if (c_here && warp == 0) {
                int act = 0, bad = 0;
                if (owns && !a.S.frozen[k_own]) shift_update(a, k_own, s_c, M, tol2, act, bad);
                act = __popc(__ballot_sync(0xffffffffu, act));
                bad = __any_sync(0xffffffffu, bad);
                if (lane == 0) { s_flag[0] = act; s_flag[1] = bad; }
            }
            // all warps apply H; with a deferred phase C the unit order is
            // rotated so that warp 0 takes the last place in each round and,
            // when the rounds do not come out even, one unit fewer
            const int wi = c_here ? (warp + kWarps - 1) % kWarps : warp;
            const int64_t a_first = Apply::kMap == kMapStrided ? (int64_t)cta + (int64_t)G * wi : ubeg + wi;
            if constexpr (HasTwoPass<Apply>::value) {
                // two passes over the units in two orders, a grid barrier between
                for (int64_t u = a_first; u < u_end; u += u_step) ap.pass1(u, lane, zs, bp, (const V*)a.r, a.q);
                if (!grid_barrier(a.sync, epoch)) return;
                for (int64_t u = a_first; u < u_end; u += u_step) {
                    int64_t row;
                    V qn;
                    if (ap.pass2(u, lane, (const V*)a.r, a.q, row, qn)) acc_bil(rq[0], rq[1], a.r[row], qn);
                }
            } else {
                for (int64_t u = a_first; u < u_end; u += u_step) {
                    int64_t row;
                    V w;
                    if (ap(u, lane, zs, (const V*)a.r, row, w)) {
                        const V qn = vcfma(bp, a.q[row], w);
                        a.q[row] = qn;
                        acc_bil(rq[0], rq[1], a.r[row], qn);
                    }
                }
            }
            block_sum_n<2>(rq, s.scratch, s_part);
            pending = false;
            if (tid == 0) {
                double* pa = a.partA + cta;            // value-major
                pa[0] = s_part[0]; pa[G] = s_part[1];
                pa[2 * G] = (double)s_flag[0];   // unconverged shifts of this CTA after the last phase C
                pa[3 * G] = (double)s_flag[1];   // a pi^k of this CTA became zero or non-finite
            }
        }
        skip_a = false;
        SCOCG_TRACE(2);
        SCOCG_MARK(0);
        if (!grid_barrier(a.sync, epoch, a.debug_inject == 1 && cta == 0 && s.n == 3)) return;
        SCOCG_TRACE(3);
        SCOCG_MARK(1);
        grid_sum_vm1(a.partA, 4, s.red, G);
        if (tid == 0) {
            const double2 rq = c2(s.red[0], s.red[1]);
            const int active = s.n == 0 ? a.K : (int)s.red[2];
            int st = kGoOn;
            if (s.n > 0 && s.red[3] != 0.0) st = SCOCG_ERR_BREAKDOWN;
            else if (active == 0) st = SCOCG_OK;
            else if (s.n >= a.max_iter) st = SCOCG_NOT_CONVERGED;
            else if (cabs2(s.rho) == 0.0 || cabs2(rq) == 0.0 || !cfinite(rq)) st = SCOCG_ERR_BREAKDOWN;
            else {
                s.alpha = cdiv(s.rho, rq);
                if (a.debug_inject == 2 && s.n == 3) s.alpha = c2(__longlong_as_double(0x7ff8000000000000ll), 0);
                if (!cfinite(s.alpha)) st = SCOCG_ERR_BREAKDOWN;
                s_vs[2] = Vec<R>::make(s.alpha);
                s.shift_iters += active;
            }
            s.active = active;
            s_flag[2] = st;
        }
        __syncthreads();
        SCOCG_MARK(6);
        if (s_flag[2] != kGoOn) { status = s_flag[2]; break; }

        // ---- full-vector mode: this iteration's shift scalars for all shifts
        // (every CTA computes them, with the same arithmetic as phase C)
        if constexpr (kFull) {
            if (a.Xf) {
                double2* s_inv = s_full;
                double2* s_bet = s_full + a.K;
                double2* s_alp = s_full + 2 * a.K;
                int* s_act = reinterpret_cast<int*>(s_full + 3 * a.K);
                const double2 t2 = cdiv(cmul(s.alpha, s.beta_prev), s.alpha_prev);
                for (int k = tid; k < a.K; k += kBlock) {
                    int act = 0;
                    if (!__ldcg(a.S.frozen + k)) {
                        const double2 pp = __ldcg(a.S.pi_prev + k), pc = __ldcg(a.S.pi_cur + k);
                        const double2 ic = __ldcg(a.S.inv_cur + k);
                        const double2 ratio = cmul(pp, ic);
                        const double2 pn = cadd(cmul(cadd(c2(1, 0), cmul(s.alpha, __ldcg(a.S.sigma + k))), pc),
                                                cmul(t2, csub(pc, pp)));
                        const double2 in = crecip(pn);
                        s_inv[k] = ic;
                        s_bet[k] = cmul(cmul(ratio, ratio), s.beta_prev);
                        s_alp[k] = cmul(cmul(pc, in), s.alpha);
                        act = 1;
                    }
                    s_act[k] = act;
                }
                __syncthreads();
            }
        }

        // ---- phase B: r_{n+1} = r_n - alpha_n q_n; partials rho, ||r||^2, c^T r
        {
            const V al = s_vs[2];
            const V bp = s_vs[1];
            const bool track_x = kMixed && s.replace_on;
            bool plain = !track_x;
            if constexpr (kFull) plain = plain && a.Xf == nullptr;
            AT acc[5] = {};
            if (plain) {
                // one row ahead: the next row's loads are in flight while this
                // row is updated and stored (same rows, same order per thread)
                int64_t i = rbeg + tid;
                V ro = vzero<V>(), qo = vzero<V>(), co = vzero<V>();
                if (i < rend) { ro = a.r[i]; qo = a.q[i]; if (a.cvec) co = a.cvec[i]; }
                for (; i < rend; i += kBlock) {
                    const int64_t inx = i + kBlock;
                    V r1 = vzero<V>(), q1 = vzero<V>(), c1 = vzero<V>();
                    if (inx < rend) { r1 = a.r[inx]; q1 = a.q[inx]; if (a.cvec) c1 = a.cvec[inx]; }
                    const V rn = r_update(ro, al, qo);
                    a.r[i] = rn;
                    acc_r<R>(acc, rn, a.cvec ? &co : nullptr);
                    ro = r1; qo = q1; co = c1;
                }
            }
            for (int64_t i = rbeg + tid; !plain && i < rend; i += kBlock) {
                const V ro = a.r[i];
                if constexpr (kFull) {
                    if (a.Xf) {
                        // p^k_n = r_n / pi^k_n + beta^k_{n-1} p^k_{n-1};  x^k_{n+1} = x^k_n + alpha^k_n p^k_n
                        const int* s_act = reinterpret_cast<const int*>(s_full + 3 * a.K);
                        const double2 rw = Vec<R>::wide(ro);
                        for (int k = 0; k < a.K; ++k) {
                            if (!s_act[k]) continue;
                            const size_t o = (size_t)k * a.n + i;
                            const double2 p = vcfma(s_full[a.K + k], a.Pf[o], cmul(rw, s_full[k]));
                            a.Pf[o] = p;
                            a.Xf[o] = vcfma(s_full[2 * a.K + k], p, a.Xf[o]);
                        }
                    }
                }
                if constexpr (kMixed) {
                    if (track_x) {
                        // p_n = r_n + beta_{n-1} p_{n-1};  x_{n+1} = x_n + alpha_n p_n (compensated sum)
                        const V p = vcfma(bp, a.p_seed[i], ro);
                        a.p_seed[i] = p;
                        const V inc = vcfma(al, p, vzero<V>());
                        const V hi = a.x_hi[i];
                        V lo = a.x_lo[i];
                        const float sx = hi.x + inc.x, bx = sx - hi.x;
                        const float sy = hi.y + inc.y, by = sy - hi.y;
                        lo.x += (hi.x - (sx - bx)) + (inc.x - bx);
                        lo.y += (hi.y - (sy - by)) + (inc.y - by);
                        a.x_hi[i] = make_float2(sx, sy);
                        a.x_lo[i] = lo;
                    }
                }
                const V rn = r_update(ro, al, a.q[i]);
                a.r[i] = rn;
                acc_r<R>(acc, rn, a.cvec ? a.cvec + i : nullptr);
            }
            __syncthreads();
            finish_r_partials(a, acc, rbeg, rend, s, s_part, myB, G);
        }
        SCOCG_TRACE(4);
        SCOCG_MARK(2);
        if (!grid_barrier(a.sync, epoch)) return;
        SCOCG_TRACE(5);
        SCOCG_MARK(3);
        grid_sum_vm1(a.partB, nred, s.red, G);
        SCOCG_MARK(5);
        // the scalars of this iteration: independent FP64 divisions and roots
        // run in three warps at once
        if (tid < M) {
            s.cr_next[tid] = dense_proj ? c2(s.red[3 + 2 * tid], s.red[4 + 2 * tid])
                                        : (chk(a.dbg, 12, a.cidx[tid], a.n) ? Vec<R>::wide(__ldcg(a.r + a.cidx[tid])) : c2(0, 0));
            s_c.cr[tid] = s.cr_cur[tid];
        }
        if (tid == 0) {
            s.t2 = cdiv(cmul(s.alpha, s.beta_prev), s.alpha_prev);
            s_c.alpha = s.alpha; s_c.beta_prev = s.beta_prev; s_c.t2 = s.t2; s_c.n = s.n;
        } else if (tid == 32) {
            s.rnorm_next = sqrt(s.red[2]);
            s.rn_b = s.rnorm_next / s.bnorm;
            s_c.rn_b2 = s.rn_b * s.rn_b;
            s_flag[4] = a.tol > 0.0 && s_c.rn_b2 <= tol2;    // the seed (pi = 1) has converged
        } else if (tid == 64) {
            s.beta_next = cdiv(c2(s.red[0], s.red[1]), s.rho);
        }
        __syncthreads();

        // ---- phase C: per-shift scalar recurrences for this CTA's shifts
        // (one complex reciprocal per shift; 1/pi^k_n is carried between
        // iterations and residuals are compared squared), here or deferred
        const bool seed_conv = s_flag[4] != 0;
        const bool defer = defer_ok && !seed_conv;
        if (!defer) {
            int my_active = 0, my_bad = 0;
            if (owns && !a.S.frozen[k_own]) shift_update(a, k_own, s_c, M, tol2, my_active, my_bad);
            const int cnt_active = __syncthreads_count(my_active);
            const int any_bad = __syncthreads_or(my_bad);
            if (tid == 0) { s_flag[0] = cnt_active; s_flag[1] = any_bad; }
        }
        pending = defer;
        if (tid == 0) {
            s.beta_prev = s.beta_next;
            s_vs[1] = Vec<R>::make(s.beta_prev);
            s.alpha_prev = s.alpha;
            s.rho_prev = s.rho;
            s.rho = c2(s.red[0], s.red[1]);
            s.rnorm = s.rnorm_next;
            s.n += 1;
        }
        if (tid < M) s.cr_cur[tid] = s.cr_next[tid];
        __syncthreads();

        // ---- seed switching (Sec. III.C) once the seed has converged
        SCOCG_TRACE(6);
        SCOCG_MARK(4);
        if (seed_conv) {
            SCOCG_TRACE(7);
            // local candidate: the unconverged shift with the smallest |pi| (largest residual)
            double best = INFINITY;
            int arg = 0x7fffffff;
            if (owns && !a.S.frozen[k_own]) { best = -cabs2(a.S.inv_cur[k_own]); arg = k_own; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
                if (ob < best || (ob == best && oa < arg)) { best = ob; arg = oa; }
            }
            if (lane == 0) { s_min[warp] = best; s_arg[warp] = arg; }
            __syncthreads();
            if (tid == 0) {
                for (int w = 1; w < kWarps; ++w)
                    if (s_min[w] < best || (s_min[w] == best && s_arg[w] < arg)) { best = s_min[w]; arg = s_arg[w]; }
                // the candidate's recurrence values travel with it, so that no CTA
                // reads them after their owner has rebased them below
                double* pc = a.partC + (size_t)cta * kPartC;
                pc[0] = (double)s_flag[0]; pc[1] = best; pc[2] = (double)arg; pc[3] = (double)s_flag[1];
                if (arg < a.K && chk(a.dbg, 10, arg, a.K)) {
                    const double2 pp = a.S.pi_prev[arg], pq = a.S.pi_cur[arg], ak = a.S.alpha_k[arg];
                    pc[4] = pp.x; pc[5] = pp.y; pc[6] = pq.x; pc[7] = pq.y; pc[8] = ak.x; pc[9] = ak.y;
                }
            }
            SCOCG_TRACE(8);
            if (!grid_barrier(a.sync, epoch)) return;
            SCOCG_TRACE(9);
            __shared__ double s_sw[6];
            if (tid == 0) {
                double tot = 0, bad = 0, gbest = INFINITY;
                int garg = 0x7fffffff, gc = -1;
                for (int c = 0; c < G; ++c) {
                    const double* pc = a.partC + (size_t)c * kPartC;
                    tot += __ldcg(pc); bad += __ldcg(pc + 3);
                    const double b2 = __ldcg(pc + 1);
                    const int a2 = (int)__ldcg(pc + 2);
                    if (b2 < gbest || (b2 == gbest && a2 < garg)) { gbest = b2; garg = a2; gc = c; }
                }
                int st = kGoOn;
                if (bad != 0.0) st = SCOCG_ERR_BREAKDOWN;
                else if (tot == 0.0) st = SCOCG_OK;
                else if (!a.allow_switch) st = SCOCG_ERR_BREAKDOWN;
                else if (gc < 0 || !chk(a.dbg, 11, garg, a.K)) st = SCOCG_ERR_BREAKDOWN;
                else
                    for (int j = 0; j < 6; ++j) s_sw[j] = __ldcg(a.partC + (size_t)gc * kPartC + 4 + j);
                s_flag[2] = st;
                s_flag[3] = garg;
            }
            __syncthreads();
            if (s_flag[2] != kGoOn) { status = s_flag[2]; break; }
            const int s2 = s_flag[3];
            SCOCG_TRACE(10 + 100 * s2);
            const double2 pin = c2(s_sw[0], s_sw[1]);        // pi^{s'}_n
            const double2 pin1 = c2(s_sw[2], s_sw[3]);       // pi^{s'}_{n+1}
            const double2 alpha_s2 = c2(s_sw[4], s_sw[5]);   // alpha^{s'}_n
            // r' = r_{n+1} / pi'_{n+1};  q' = (r_n / pi'_n - r_{n+1} / pi'_{n+1}) / alpha'_n,
            // with r_n = r_{n+1} + alpha_n q_n
            const double2 inv1 = cdiv(c2(1, 0), pin1);
            const double2 ca = cdiv(csub(cdiv(c2(1, 0), pin), inv1), alpha_s2);   // times r_{n+1}
            const double2 cb = cdiv(cdiv(s.alpha_prev, pin), alpha_s2);           // times q_n
            const V v_inv1 = Vec<R>::make(inv1), v_ca = Vec<R>::make(ca), v_cb = Vec<R>::make(cb);
            for (int64_t i = rbeg + tid; i < rend; i += kBlock) {
                const V ri = a.r[i], qi = a.q[i];
                a.q[i] = vcfma(v_cb, qi, vcfma(v_ca, ri, vzero<V>()));
                a.r[i] = vcfma(v_inv1, ri, vzero<V>());
            }
            SCOCG_TRACE(11);
            if (owns && chk(a.dbg, 13, s2, a.K)) {
                const int k = k_own;
                if (k == s2) {
                    a.S.pi_prev[k] = c2(1, 0); a.S.pi_cur[k] = c2(1, 0); a.S.inv_cur[k] = c2(1, 0);
                } else {
                    a.S.pi_prev[k] = cdiv(a.S.pi_prev[k], pin);
                    a.S.pi_cur[k] = cdiv(a.S.pi_cur[k], pin1);
                    a.S.inv_cur[k] = cmul(a.S.inv_cur[k], pin1);
                }
                a.S.sigma[k] = csub(a.z[k], a.z[s2]);
            }
            __syncthreads();
            if (tid == 0) {
                const double2 ratio = cdiv(pin, pin1);
                s.rho = cdiv(s.rho, cmul(pin1, pin1));
                s.beta_prev = cmul(cmul(ratio, ratio), s.beta_prev);
                s.alpha_prev = alpha_s2;
                s.rnorm = s.rnorm / cabs_(pin1);
                s.seed = s2;
                s.zs = a.z[s2];
                s_vs[0] = Vec<R>::make(s.zs);
                s_vs[1] = Vec<R>::make(s.beta_prev);
                s.n_switch += 1;
                s.replace_on = 0;        // the new seed's full solution is not tracked
            }
            if (tid < M) s.cr_cur[tid] = cmul(s.cr_cur[tid], inv1);
            SCOCG_TRACE(12);
            if (!grid_barrier(a.sync, epoch)) return;
            SCOCG_TRACE(13);
        }

        // ---- MIXED: FP64 true-residual replacement r_{n+1} = b - (z_s - H) x_{n+1}
        if constexpr (kMixed) {
            if (s.replace_on && s.n % a.replace_every == 0) {
                for (int64_t i = rbeg + tid; i < rend; i += kBlock) {
                    const V hi = a.x_hi[i], lo = a.x_lo[i];
                    a.xd[i] = c2((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y);
                }
                if (!grid_barrier(a.sync, epoch)) return;
                const double2 zs = s.zs;
                for (int64_t u = u_first; u < u_end; u += u_step) {
                    int64_t row;
                    double2 w;
                    if (ap(u, lane, zs, (const double2*)a.xd, row, w)) {
                        const double2 bi = a.b[row];
                        a.r[row] = Vec<R>::make(c2(bi.x - w.x, bi.y - w.y));
                    }
                }
                if (!grid_barrier(a.sync, epoch)) return;
                r_partials(a, rbeg, rend, s, s_part, myB, G);
                if (!grid_barrier(a.sync, epoch)) return;
                grid_sum_vm1(a.partB, nred, s.red, G);
                if (tid == 0) {
                    s.rho = c2(s.red[0], s.red[1]);
                    s.beta_prev = cdiv(s.rho, s.rho_prev);
                    s_vs[1] = Vec<R>::make(s.beta_prev);
                    s.rnorm = sqrt(s.red[2]);
                    s.n_replace += 1;
                }
                if (tid < M) {
                    s.cr_cur[tid] = dense_proj ? c2(s.red[3 + 2 * tid], s.red[4 + 2 * tid])
                                               : (chk(a.dbg, 12, a.cidx[tid], a.n) ? Vec<R>::wide(__ldcg(a.r + a.cidx[tid])) : c2(0, 0));
                }
                __syncthreads();
            }
        }
    }

    // ------------------------------------------------------------ outputs
    SCOCG_TRACE(20);
    if (owns) {
        for (int m = 0; m < M; ++m) a.G[(size_t)m * a.K + k_own] = a.S.X[(size_t)k_own * M + m];
    }
    if (cta == 0 && tid == 0) {
        // the stopping apply took the deferred shift update (and rotated its
        // units) when the iteration before had not converged the seed
        if (a.rstate) save_resume_state(a.rstate, s, status, M, defer_ok && s_flag[4] == 0);
        a.stats->iters = s.n;
        a.stats->n_switch = s.n_switch;
        a.stats->seed = s.seed;
        a.stats->n_replace = s.n_replace;
        a.stats->shift_iters = s.shift_iters;
        a.stats->status = status;
        if (status != SCOCG_OK) atomicCAS(a.sync.status, 0, status);
    }
}

// One solve on the whole grid.
// CTAs per SM the persistent kernel is compiled for: two (64 registers a
// thread) hide the latency of the FP32-pipe modes; FP64 solves are bound by
// the FP64 pipe, where one CTA per SM (128 registers, half the CTAs at every
// grid barrier) measured faster.
#ifndef SCOCG_DF_CTAS_PER_SM
#define SCOCG_DF_CTAS_PER_SM 2
#endif
template <typename R> struct MinBlocks { static constexpr int value = 2; };
template <> struct MinBlocks<double> { static constexpr int value = 1; };
template <> struct MinBlocks<DF> { static constexpr int value = SCOCG_DF_CTAS_PER_SM; };

template <typename R, class Apply, bool kResume = false>
__global__ void __launch_bounds__(kBlock, MinBlocks<R>::value) cocg_persistent(SolveArgs<R> a, Apply ap) {
    cocg_body<R, Apply, kResume>(a, ap, (int)gridDim.x, (int)blockIdx.x);
}

// Several independent solves in one launch: CTAs [cta_off[s], cta_off[s+1])
// run system s with its own arguments, barrier counter and partials.
template <typename R, class Apply>
__global__ void __launch_bounds__(kBlock, 2) cocg_multi(const SolveArgs<R>* args, const Apply* aps,
                                                        const int* cta_off, int nsys) {
    int sys = 0;
    while (sys + 1 < nsys && cta_off[sys + 1] <= (int)blockIdx.x) ++sys;
    const SolveArgs<R> a = args[sys];
    const Apply ap = aps[sys];
    cocg_body(a, ap, cta_off[sys + 1] - cta_off[sys], (int)blockIdx.x - cta_off[sys]);
}

}  // namespace scocg
