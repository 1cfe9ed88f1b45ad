// Host driver of the multi-right-hand-side (block) shifted-COCG kernel, and the
// autotuner that picks its slot count T and grid for a handle.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "block_kernel.cuh"
#include "solver_launch.h"

namespace scocg {
namespace {

template <typename R, int T>
int block_occupancy() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cocg_block<R, T>, kBlock, 0) != cudaSuccess) return 0;
    return nb;
}

template <typename R, int T>
int run_block(scocg_ctx* h, const scocg_c128* shifts, int K, const void* rhs, int nrhs, const int64_t* proj_idx,
              int M, double tol, scocg_c128* G_out, scocg_info* info, int ctas_per_sm, int max_iter, int prec) {
    using V = typename Vec<R>::T;
    using W = typename ValT<R>::T;
    const int occ = block_occupancy<R, T>();
    if (occ <= 0) return SCOCG_ERR_CUDA;
    const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
    const int64_t n = h->n;
    const int npairs = T * K;
    constexpr int RPW = 32 / T;
    // at least eight warp steps of rows per warp, and one thread per (slot, shift) pair
    int64_t want = std::max<int64_t>((n + 8 * kWarps * RPW - 1) / (8 * kWarps * RPW), (npairs + kBlock - 1) / kBlock);
    if (h->opts.grid > 0) want = h->opts.grid;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per_sm * h->num_sms));

    const size_t vbytes = sizeof(V) * (size_t)n * T;
    const size_t P1 = (size_t)npairs;
    BlockArgs<R> a{};
    int64_t* d_cidx = nullptr;
    double2* d_z = nullptr;
    auto carve = [&](Carver& c) {
        a.r = (V*)c.take(vbytes);
        a.q = (V*)c.take(vbytes);
        d_cidx = (int64_t*)c.take(sizeof(int64_t) * (size_t)nrhs * M);
        d_z = (double2*)c.take(sizeof(double2) * K);
        a.pi_prev = (double2*)c.take(sizeof(double2) * P1);
        a.pi_cur = (double2*)c.take(sizeof(double2) * P1);
        a.sigma = (double2*)c.take(sizeof(double2) * P1);
        a.alpha_k = (double2*)c.take(sizeof(double2) * P1);
        a.inv_cur = (double2*)c.take(sizeof(double2) * P1);
        a.P = (double2*)c.take(sizeof(double2) * P1 * M);
        a.X = (double2*)c.take(sizeof(double2) * P1 * M);
        a.frozen = (int*)c.take(sizeof(int) * P1);
        a.iters = (int*)c.take(sizeof(int) * P1);
        a.resid = (double*)c.take(sizeof(double) * P1);
        a.out_iters = (int*)c.take(sizeof(int) * (size_t)nrhs * K);
        a.out_resid = (double*)c.take(sizeof(double) * (size_t)nrhs * K);
        a.out_info = (int*)c.take(sizeof(int) * 4 * (size_t)nrhs);
        a.partA = (double*)c.take(sizeof(double) * kNvA * T * grid);
        a.partB = (double*)c.take(sizeof(double) * kNvB * T * grid);
        a.partC = (double*)c.take(sizeof(double) * kNvC * T * grid);
        a.res = (double*)c.take(sizeof(double) * (kNvA > kNvB ? kNvA : kNvB) * T);
    };
    Carver measure{nullptr, 0};
    carve(measure);
    cudaError_t e = h->ws.reserve(measure.off);
    if (e != cudaSuccess) return cuda_status(e);
    Carver cut{static_cast<char*>(h->ws.base), 0};
    carve(cut);
    cudaStream_t st = h->stream;
    e = cudaMemcpyAsync(d_z, shifts, sizeof(double2) * K, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_cidx, proj_idx, sizeof(int64_t) * (size_t)nrhs * M, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_ctrl, 0, sizeof(Ctrl), st);
    if (e != cudaSuccess) return cuda_status(e);

    a.n = n;
    a.nnz = h->nnz;
    a.rowptr = h->d_rowptr;
    a.col = h->d_col;
    if constexpr (std::is_same<W, double>::value) a.val = h->d_val64;
    else a.val = h->d_val32;
    // the 4x4-blocked layout, when the handle has it: each gathered row of x
    // then serves the four rows of a block row
    const bool blocked = h->bsr_ok && h->d_unit_off && h->n % 4 == 0;
    a.unit_off = blocked ? h->d_unit_off : nullptr;
    a.bcol = blocked ? h->d_bcol : nullptr;
    if constexpr (std::is_same<W, double>::value) a.bval = blocked ? h->d_bval64 : nullptr;
    else a.bval = blocked ? h->d_bval32 : nullptr;
    a.nslots = blocked ? h->nslots : 0;
    a.b = static_cast<const double2*>(rhs);
    a.nrhs = nrhs;
    a.cidx = d_cidx;
    a.nproj = M;
    a.K = K;
    a.z = d_z;
    a.seed0 = (h->opts.seed >= 0 && h->opts.seed < K) ? h->opts.seed : default_seed(shifts, K);
    a.allow_switch = !h->opts.no_switch;
    a.tol = tol;
    a.max_iter = max_iter;
    a.G = reinterpret_cast<double2*>(G_out);
    a.sync.count = &h->d_ctrl->count;
    a.sync.status = &h->d_ctrl->status;
    a.sync.timeout_ns = (uint64_t)(h->opts.timeout_ms * 1e6);
    a.sync.nctas = grid;
    a.stats = &h->d_ctrl->stats;
    a.dbg = h->d_ctrl->dbg;
    a.phase_ns = nullptr;
#ifdef SCOCG_PHASE_TIMERS
    static unsigned long long* h_ns = nullptr;
    static int h_ns_n = 0;
    if (h_ns_n < grid) {
        if (h_ns) cudaFreeHost(h_ns);
        h_ns = nullptr; h_ns_n = 0;
        if (cudaHostAlloc((void**)&h_ns, sizeof(unsigned long long) * 8 * grid, cudaHostAllocMapped) == cudaSuccess)
            h_ns_n = grid;
    }
    if (h_ns) {
        std::memset(h_ns, 0, sizeof(unsigned long long) * 8 * grid);
        cudaHostGetDevicePointer((void**)&a.phase_ns, h_ns, 0);
    }
#endif

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEventCreate(&ev0); cudaEventCreate(&ev1);
    cudaEventRecord(ev0, st);
    void* args[] = {(void*)&a};
    e = cudaLaunchCooperativeKernel((const void*)cocg_block<R, T>, dim3(grid), dim3(kBlock), args, 0, st);
    cudaEventRecord(ev1, st);
    Ctrl c;
    std::vector<int> oinfo(4 * (size_t)nrhs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c, h->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(oinfo.data(), a.out_info, sizeof(int) * oinfo.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && info && info->freeze_iter)
        e = cudaMemcpyAsync(info->freeze_iter, a.out_iters, sizeof(int) * (size_t)nrhs * K, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && info && info->resid)
        e = cudaMemcpyAsync(info->resid, a.out_resid, sizeof(double) * (size_t)nrhs * K, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0); cudaEventDestroy(ev1);
    if (e != cudaSuccess) return cuda_status(e);
#ifdef SCOCG_PHASE_TIMERS
    if (h_ns) {
        double tot[8] = {0};
        for (int cc = 0; cc < grid; ++cc)
            for (int k = 0; k < 8; ++k) tot[k] += (double)((volatile unsigned long long*)h_ns)[8 * cc + k];
        std::fprintf(stderr,
                     "scocg block T=%d grid %d phase ms (CTA average): A %.3f bar1 %.3f decide %.3f B %.3f bar2 %.3f "
                     "red2 %.3f C %.3f switch+top %.3f\n", T, grid,
                     tot[0] / grid * 1e-6, tot[1] / grid * 1e-6, tot[6] / grid * 1e-6, tot[2] / grid * 1e-6,
                     tot[3] / grid * 1e-6, tot[5] / grid * 1e-6, tot[4] / grid * 1e-6, tot[7] / grid * 1e-6);
        // spread of the apply time over the CTAs (first and last CTA ids of the extremes)
        double mn = 1e300, mx = 0.0;
        int cmn = 0, cmx = 0;
        for (int cc = 0; cc < grid; ++cc) {
            const double v = (double)((volatile unsigned long long*)h_ns)[8 * cc];
            if (v < mn) { mn = v; cmn = cc; }
            if (v > mx) { mx = v; cmx = cc; }
        }
        std::fprintf(stderr, "scocg block apply per CTA ms: min %.3f (cta %d) max %.3f (cta %d)\n", mn * 1e-6, cmn,
                     mx * 1e-6, cmx);
    }
#endif
    if (c.dbg[0]) {
        std::fprintf(stderr, "scocg checked build: out-of-range index at site %llu: %lld (limit %lld)\n", c.dbg[1],
                     (long long)c.dbg[2], (long long)c.dbg[3]);
        return SCOCG_ERR_INVALID;
    }
    if (c.status < 0) return c.status;   // barrier timeout or another device-side failure
    int worst = SCOCG_OK, iters = 0, nsw = 0;
    for (int j = 0; j < nrhs; ++j) {
        const int sj = oinfo[4 * j];
        if (sj < 0 && worst >= 0) worst = sj;
        else if (sj == SCOCG_NOT_CONVERGED && worst == SCOCG_OK) worst = sj;
        iters = std::max(iters, oinfo[4 * j + 1]);
        nsw += oinfo[4 * j + 2];
    }
    if (info) {
        if (info->resid)   // the kernel keeps squared residual estimates
            for (size_t j = 0; j < (size_t)nrhs * K; ++j) info->resid[j] = std::sqrt(info->resid[j]);
        info->iters = c.stats.iters;
        info->n_switch = nsw;
        info->seed_final = oinfo[4 * (nrhs - 1) + 3];
        info->n_replace = 0;
        info->shift_iters = c.stats.shift_iters;
        info->seconds = ms * 1e-3;
        // one block iteration: H once in the layout used, six passes over the [n][T] vectors
        const double vb = prec == SCOCG_MIXED ? 8.0 : 16.0;
        const double hb = blocked ? (double)h->nslots * 8 * (4.0 + 16.0 * sizeof(W)) + 4.0 * (h->nunits_bsr + 1)
                                  : (double)h->nnz * (4.0 + sizeof(W)) + 4.0 * (n + 1);
        info->bytes_per_iter = hb + 6.0 * vb * (double)n * T;
    }
    return worst;
}

template <typename R>
int run_block_t(int T, scocg_ctx* h, const scocg_c128* shifts, int K, const void* rhs, int nrhs,
                const int64_t* proj_idx, int M, double tol, scocg_c128* G_out, scocg_info* info, int per_sm,
                int max_iter, int prec) {
    switch (T) {
        case 8: return run_block<R, 8>(h, shifts, K, rhs, nrhs, proj_idx, M, tol, G_out, info, per_sm, max_iter, prec);
        case 16: return run_block<R, 16>(h, shifts, K, rhs, nrhs, proj_idx, M, tol, G_out, info, per_sm, max_iter, prec);
        case 32: return run_block<R, 32>(h, shifts, K, rhs, nrhs, proj_idx, M, tol, G_out, info, per_sm, max_iter, prec);
    }
    return SCOCG_ERR_INVALID;
}

int run_any(int prec, int T, scocg_ctx* h, const scocg_c128* shifts, int K, const void* rhs, int nrhs,
            const int64_t* proj_idx, int M, double tol, scocg_c128* G_out, scocg_info* info, int per_sm,
            int max_iter) {
    if (prec == SCOCG_MIXED)
        return run_block_t<float>(T, h, shifts, K, rhs, nrhs, proj_idx, M, tol, G_out, info, per_sm, max_iter, prec);
    if (prec == SCOCG_MIXED_DF)
        return run_block_t<DF>(T, h, shifts, K, rhs, nrhs, proj_idx, M, tol, G_out, info, per_sm, max_iter, prec);
    return run_block_t<double>(T, h, shifts, K, rhs, nrhs, proj_idx, M, tol, G_out, info, per_sm, max_iter, prec);
}

}  // namespace

// Default slot count: the smallest T in {8, 16, 32} that holds every
// right-hand side, else 32.
int block_default_tile(int nrhs) { return nrhs <= 8 ? 8 : (nrhs <= 16 ? 16 : 32); }

int block_solve(scocg_ctx* h, const scocg_c128* shifts, int K, const void* rhs, int nrhs, const int64_t* proj_idx,
                int M, double tol, scocg_c128* G_out, scocg_info* info, int prec, int T, int per_sm) {
    return run_any(prec, T, h, shifts, K, rhs, nrhs, proj_idx, M, tol, G_out, info, per_sm, h->opts.max_iter);
}

// The autotuner: time a short solve (a bounded number of block iterations on
// the first right-hand sides) for every candidate (T, CTAs per SM) and keep
// the fastest per shift-iteration.  The choice is cached in the handle for
// (precision, nshift, nproj, min(nrhs, 32)).
int block_autotune(scocg_ctx* h, const scocg_c128* shifts, int K, const void* rhs, int nrhs,
                   const int64_t* proj_idx, int M, double tol, scocg_c128* G_out, int prec, int* T_out,
                   int* per_sm_out) {
    const int key_rhs = std::min(nrhs, 32);
    for (const TuneEntry& t : h->tune)
        if (t.prec == prec && t.K == K && t.M == M && t.nrhs == key_rhs) {
            *T_out = t.T; *per_sm_out = t.per_sm;
            return SCOCG_OK;
        }
    const int tiles[3] = {8, 16, 32};
    const int trial_iters = 24;
    double best = INFINITY;
    int bestT = block_default_tile(nrhs), best_sm = 0;
    for (int T : tiles) {
        if (T > 8 && T / 2 >= nrhs) break;            // slots that could never fill
        for (int per_sm = 1; per_sm <= 2; ++per_sm) {
            const int ntrial = std::min(nrhs, T);
            scocg_info inf{};
            const int st = run_any(prec, T, h, shifts, K, rhs, ntrial, proj_idx, M, tol, G_out, &inf, per_sm,
                                   trial_iters);
            if (st < 0 && st != SCOCG_ERR_BREAKDOWN) return st;
            if (inf.shift_iters <= 0 || inf.seconds <= 0.0) continue;
            const double cost = inf.seconds / (double)inf.shift_iters;
            if (cost < best) { best = cost; bestT = T; best_sm = per_sm; }
        }
    }
    h->tune.push_back(TuneEntry{prec, K, M, key_rhs, bestT, best_sm});
    *T_out = bestT;
    *per_sm_out = best_sm;
    return SCOCG_OK;
}

}  // namespace scocg
