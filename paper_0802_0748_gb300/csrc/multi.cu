// Several independent shifted-COCG solves in one cooperative launch (the
// multi-system work list).  The co-resident CTAs are split among the systems:
// each gets at least enough CTAs for its shifts and otherwise a share
// proportional to its rows; each system keeps its own arguments, barrier
// counter, partials and scalars (cocg_multi in solver_kernel.cuh).  The
// control-block resets and the launch can be captured into a CUDA graph and
// replayed while sizes and buffers stay the same.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "solver_kernel.cuh"

namespace scocg {
namespace {

template <typename R, class Apply>
int multi_occupancy() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cocg_multi<R, Apply>, kBlock, 0) != cudaSuccess) return 0;
    return nb;
}

template <typename W>
const W* pick_vals(const Layout& L, bool blocked);
template <> const double* pick_vals<double>(const Layout& L, bool blocked) { return blocked ? L.bval64 : L.val64; }
template <> const float* pick_vals<float>(const Layout& L, bool blocked) { return blocked ? L.bval32 : L.val32; }

template <typename W, class Apply> Apply make_apply(const Layout& L);
template <> ApplyBSR4<double> make_apply<double, ApplyBSR4<double>>(const Layout& L) {
    return ApplyBSR4<double>{L.unit_off, L.bcol, L.bval64, L.n, L.nslots, nullptr};
}
template <> ApplyBSR4C<float> make_apply<float, ApplyBSR4C<float>>(const Layout& L) {
    return ApplyBSR4C<float>{L.unit_off, L.bcol, L.bval32c, L.n, L.nslots, nullptr};
}
template <> ApplyBSR4<float> make_apply<float, ApplyBSR4<float>>(const Layout& L) {
    return ApplyBSR4<float>{L.unit_off, L.bcol, L.bval32, L.n, L.nslots, nullptr};
}
template <typename W, int LPR>
ApplyCSR<W, LPR> make_csr(const Layout& L) { return ApplyCSR<W, LPR>{L.rowptr, L.col, pick_vals<W>(L, false), L.n, L.nnz, nullptr}; }

__global__ void k_to_c64m(int64_t n, const double2* in, float2* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
__global__ void k_to_dfm(int64_t n, const double2* in, float4* out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = df_from(in[i]);
}

// Per-system state kept between calls (graph replay needs stable buffers).
struct SysPlan {
    int grid = 0;
    int K = 0, M = 0;
    void* cvec = nullptr;      // projection vectors converted to the vector precision
    int64_t* cidx = nullptr;   // unit projections
    double2* z = nullptr;
    ShiftState S{};
};

}  // namespace

struct MultiPlan {
    std::vector<scocg_ctx*> hs;
    std::vector<unsigned long long> gens;   // workspace generation of each handle when planned
    std::vector<int> nshift, nproj;
    std::vector<const void*> rhs, pvec;
    std::vector<const int64_t*> pidx;
    std::vector<scocg_c128*> G;
    double tol = 0;
    int prec = 0;
    int kind = -1;
    std::vector<SysPlan> sys;
    void* d_args = nullptr;    // [nsys] SolveArgs<R>
    void* d_aps = nullptr;     // [nsys] Apply
    int* d_off = nullptr;      // [nsys + 1]
    int total_grid = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t cap = nullptr;   // capture stream (the handles' stream may be the legacy default stream)

    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        cap = nullptr;
        cudaFree(d_args); cudaFree(d_aps); cudaFree(d_off);
        exec = nullptr; graph = nullptr; d_args = d_aps = nullptr; d_off = nullptr;
    }
};

namespace {

MultiPlan* g_plan = nullptr;   // the most recent plan (one cached plan per process)

bool same_plan(const MultiPlan* p, int nsys, const scocg_handle* hs, const int* nshift, const void* const* rhs,
               const void* const* pvec, const int64_t* const* pidx, const int* nproj, double tol,
               scocg_c128* const* G, int prec) {
    if (!p || (int)p->hs.size() != nsys || p->tol != tol || p->prec != prec) return false;
    for (int s = 0; s < nsys; ++s) {
        if (p->hs[s] != hs[s] || p->gens[s] != hs[s]->ws_gen || p->nshift[s] != nshift[s] || p->rhs[s] != rhs[s] ||
            p->nproj[s] != nproj[s] ||
            p->G[s] != G[s] || p->pvec[s] != (pvec ? pvec[s] : nullptr) || p->pidx[s] != (pidx ? pidx[s] : nullptr))
            return false;
    }
    return true;
}

template <typename R, class Apply>
int run_multi(int nsys, const scocg_handle* hs, const scocg_c128* const* shifts, const int* nshift,
              const void* const* rhs, const void* const* pvec, const int64_t* const* pidx, const int* nproj,
              double tol, scocg_c128* const* G_out, scocg_info* info, int use_graph, int prec,
              Apply (*mk)(const Layout&)) {
    using V = typename Vec<R>::T;
    scocg_ctx* h0 = hs[0];
    cudaStream_t st = h0->stream;
    const bool mixed = prec == SCOCG_MIXED, dfm = prec == SCOCG_MIXED_DF;
    const int occ = multi_occupancy<R, Apply>();
    if (occ <= 0) return SCOCG_ERR_CUDA;
    const int maxco = occ * h0->num_sms;
    cudaError_t e = cudaSuccess;

    const bool reuse = use_graph && same_plan(g_plan, nsys, hs, nshift, rhs, pvec, pidx, nproj, tol, G_out, prec);
    MultiPlan* P = g_plan;
    if (!reuse) {
        if (g_plan) { g_plan->release(); delete g_plan; }
        P = g_plan = new MultiPlan();
        P->tol = tol; P->prec = prec;
        P->sys.resize(nsys);
        // grid split: minimum per system, the rest in proportion to rows
        std::vector<int64_t> units(nsys), gmin(nsys), gmax(nsys);
        int64_t tot_units = 0, need = 0;
        for (int s = 0; s < nsys; ++s) {
            const Layout L = hs[s]->layout(false);
            const int rpu = rows_per_unit(L.kind);
            units[s] = (hs[s]->n + rpu - 1) / rpu;
            gmin[s] = std::max<int64_t>(1, (nshift[s] + kBlock - 1) / kBlock);
            gmax[s] = std::max<int64_t>(gmin[s], (units[s] + kWarps - 1) / kWarps);
            tot_units += units[s];
            need += gmin[s];
        }
        if (need > maxco) return SCOCG_ERR_INVALID;
        std::vector<int> g(nsys);
        int used = 0;
        for (int s = 0; s < nsys; ++s) {
            const int64_t share = (int64_t)((double)maxco * (double)units[s] / (double)tot_units);
            g[s] = (int)std::min<int64_t>(gmax[s], std::max<int64_t>(gmin[s], share));
            used += g[s];
        }
        while (used > maxco) {   // trim the largest shares
            int sm = 0;
            for (int s = 1; s < nsys; ++s) if (g[s] - gmin[s] > g[sm] - gmin[sm]) sm = s;
            if (g[sm] <= gmin[sm]) return SCOCG_ERR_INVALID;
            --g[sm]; --used;
        }
        std::vector<int> off(nsys + 1, 0);
        for (int s = 0; s < nsys; ++s) off[s + 1] = off[s] + g[s];
        P->total_grid = off[nsys];
        std::vector<SolveArgs<R>> args(nsys);
        std::vector<Apply> aps(nsys);
        for (int s = 0; s < nsys && e == cudaSuccess; ++s) {
            scocg_ctx* h = hs[s];
            const int64_t n = h->n;
            const int K = nshift[s], M = nproj[s];
            const int grid = g[s];
            const int strideB = 3 + 2 * M + 1;
            const size_t velem = sizeof(V);
            const size_t vbytes = velem * (size_t)n;
            SysPlan& sp = P->sys[s];
            sp.grid = grid; sp.K = K; sp.M = M;
            SolveArgs<R> a{};
            void *r = nullptr, *q = nullptr, *cv = nullptr;
            int64_t* cidx = nullptr;
            auto carve = [&](Carver& c) {
                r = c.take(vbytes); q = c.take(vbytes);
                if (mixed) {
                    a.p_seed = (V*)c.take(vbytes); a.x_hi = (V*)c.take(vbytes); a.x_lo = (V*)c.take(vbytes);
                    a.xd = (double2*)c.take(sizeof(double2) * n);
                }
                cv = (pvec && (mixed || dfm)) ? c.take(velem * (size_t)n * M) : nullptr;
                cidx = pidx ? (int64_t*)c.take(sizeof(int64_t) * M) : nullptr;
                sp.z = (double2*)c.take(sizeof(double2) * K);
                sp.S.pi_prev = (double2*)c.take(sizeof(double2) * K);
                sp.S.pi_cur = (double2*)c.take(sizeof(double2) * K);
                sp.S.sigma = (double2*)c.take(sizeof(double2) * K);
                sp.S.alpha_k = (double2*)c.take(sizeof(double2) * K);
                sp.S.inv_cur = (double2*)c.take(sizeof(double2) * K);
                sp.S.P = (double2*)c.take(sizeof(double2) * (size_t)K * M);
                sp.S.X = (double2*)c.take(sizeof(double2) * (size_t)K * M);
                sp.S.frozen = (int*)c.take(sizeof(int) * K);
                sp.S.iters = (int*)c.take(sizeof(int) * K);
                sp.S.resid = (double*)c.take(sizeof(double) * K);
                a.partA = (double*)c.take(sizeof(double) * grid * 4);
                a.partB = (double*)c.take(sizeof(double) * grid * strideB);
                a.partC = (double*)c.take(sizeof(double) * grid * kPartC);
            };
            Carver measure{nullptr, 0};
            carve(measure);
            h->rs.ok = false;   // the handle's continuation state is overwritten
            e = h->ws.reserve(measure.off);
            if (e != cudaSuccess) break;
            Carver cut{static_cast<char*>(h->ws.base), 0};
            carve(cut);
            sp.cvec = cv;
            sp.cidx = cidx;
            const Layout L = h->layout(false);
            a.n = n;
            a.rows_per_unit = rows_per_unit(L.kind);
            a.nunits = (n + a.rows_per_unit - 1) / a.rows_per_unit;
            a.r = (V*)r; a.q = (V*)q;
            a.b = (const double2*)rhs[s];
            a.cvec = pvec ? (const V*)((mixed || dfm) ? cv : pvec[s]) : nullptr;
            a.cidx = cidx;
            a.nproj = M;
            a.replace_every = h->opts.replace_every;
            a.K = K; a.z = sp.z;
            a.seed = (h->opts.seed >= 0 && h->opts.seed < K) ? h->opts.seed : default_seed(shifts[s], K);
            a.allow_switch = !h->opts.no_switch;
            a.tol = tol;
            a.max_iter = h->opts.max_iter;
            a.S = sp.S;
            a.strideB = strideB;
            a.sync.count = &h->d_ctrl->count;
            a.sync.status = &h->d_ctrl->status;
            a.sync.timeout_ns = (uint64_t)(h->opts.timeout_ms * 1e6);
            a.sync.nctas = grid;
            a.stats = &h->d_ctrl->stats;
            a.G = reinterpret_cast<double2*>(G_out[s]);
            a.dbg = h->d_ctrl->dbg;
            args[s] = a;
            aps[s] = mk(L);
            P->hs.push_back(h);
            P->gens.push_back(h->ws_gen);
            P->nshift.push_back(K);
            P->nproj.push_back(M);
            P->rhs.push_back(rhs[s]);
            P->pvec.push_back(pvec ? pvec[s] : nullptr);
            P->pidx.push_back(pidx ? pidx[s] : nullptr);
            P->G.push_back(G_out[s]);
        }
        if (e == cudaSuccess) e = cudaMalloc(&P->d_args, sizeof(SolveArgs<R>) * nsys);
        if (e == cudaSuccess) e = cudaMalloc(&P->d_aps, sizeof(Apply) * nsys);
        if (e == cudaSuccess) e = cudaMalloc(&P->d_off, sizeof(int) * (nsys + 1));
        if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_args, args.data(), sizeof(SolveArgs<R>) * nsys, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_aps, aps.data(), sizeof(Apply) * nsys, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(P->d_off, off.data(), sizeof(int) * (nsys + 1), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { g_plan->release(); delete g_plan; g_plan = nullptr; return cuda_status(e); }
    }
    // inputs staged into the workspaces every call (outside any graph): the
    // shifts may change, and another solve on the same handle may have reused
    // the workspace in between
    for (int s = 0; s < nsys && e == cudaSuccess; ++s) {
        const SysPlan& sp = P->sys[s];
        e = cudaMemcpyAsync(sp.z, shifts[s], sizeof(double2) * nshift[s], cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && pvec && (mixed || dfm)) {
            const int64_t tot = hs[s]->n * nproj[s];
            if (mixed)
                k_to_c64m<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, (const double2*)pvec[s], (float2*)sp.cvec);
            else
                k_to_dfm<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(tot, (const double2*)pvec[s], (float4*)sp.cvec);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && pidx)
            e = cudaMemcpyAsync(sp.cidx, pidx[s], sizeof(int64_t) * nproj[s], cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return cuda_status(e);

    // the launch: control blocks reset, then the cooperative kernel
    auto enqueue = [&](cudaStream_t qs) -> cudaError_t {
        cudaError_t e2 = cudaSuccess;
        for (int s = 0; s < nsys && e2 == cudaSuccess; ++s) e2 = cudaMemsetAsync(hs[s]->d_ctrl, 0, sizeof(Ctrl), qs);
        if (e2 != cudaSuccess) return e2;
        const SolveArgs<R>* da = (const SolveArgs<R>*)P->d_args;
        const Apply* dp = (const Apply*)P->d_aps;
        const int* doff = P->d_off;
        int ns = nsys;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(P->total_grid);
        cfg.blockDim = dim3(kBlock);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = qs;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, cocg_multi<R, Apply>, da, dp, doff, ns);
    };
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEventCreate(&ev0); cudaEventCreate(&ev1);
    cudaEventRecord(ev0, st);
    if (use_graph) {
        if (!P->exec) {
            // captured on a stream of the plan's own, launched on the handles' stream
            if (!P->cap) e = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t le = enqueue(P->cap);
                cudaGraph_t gr = nullptr;
                e = cudaStreamEndCapture(P->cap, &gr);
                if (le != cudaSuccess) e = le;
                if (e == cudaSuccess) { P->graph = gr; e = cudaGraphInstantiate(&P->exec, gr, 0); }
            }
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(P->exec, st);
    } else {
        e = enqueue(st);
    }
    cudaEventRecord(ev1, st);
    int worst = SCOCG_OK;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0); cudaEventDestroy(ev1);
    if (e != cudaSuccess) return cuda_status(e);
    for (int s = 0; s < nsys; ++s) {
        Ctrl c;
        e = cudaMemcpy(&c, hs[s]->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_status(e);
        const int dst = c.status;
        if (dst < 0) worst = dst;
        else if (dst == SCOCG_NOT_CONVERGED && worst == SCOCG_OK) worst = SCOCG_NOT_CONVERGED;
        if (info) {
            scocg_info& I = info[s];
            I.iters = c.stats.iters; I.n_switch = c.stats.n_switch; I.seed_final = c.stats.seed;
            I.n_replace = c.stats.n_replace; I.shift_iters = c.stats.shift_iters; I.seconds = ms * 1e-3;
            I.bytes_per_iter = hs[s]->bytes_per_iter(prec, pvec != nullptr, nproj[s]);
            const int K = nshift[s];
            if (I.freeze_iter) e = cudaMemcpy(I.freeze_iter, P->sys[s].S.iters, sizeof(int) * K, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && I.resid) {
                e = cudaMemcpy(I.resid, P->sys[s].S.resid, sizeof(double) * K, cudaMemcpyDeviceToHost);
                for (int k = 0; k < K; ++k) I.resid[k] = std::sqrt(I.resid[k]);
            }
            if (e != cudaSuccess) return cuda_status(e);
        }
    }
    return worst;
}

template <typename R>
int dispatch_layout(LayoutKind kind, int nsys, const scocg_handle* hs, const scocg_c128* const* shifts,
                    const int* nshift, const void* const* rhs, const void* const* pvec, const int64_t* const* pidx,
                    const int* nproj, double tol, scocg_c128* const* G, scocg_info* info, int use_graph, int prec) {
    using W = typename ValT<R>::T;
    switch (kind) {
        case LayoutKind::kBsr4:
            return run_multi<R, typename BsrApply<R>::T>(nsys, hs, shifts, nshift, rhs, pvec, pidx, nproj, tol, G,
                                                         info, use_graph, prec,
                                                         &make_apply<W, typename BsrApply<R>::T>);
        case LayoutKind::kCsr1:
            return run_multi<R, ApplyCSR<W, 1>>(nsys, hs, shifts, nshift, rhs, pvec, pidx, nproj, tol, G, info,
                                                use_graph, prec, &make_csr<W, 1>);
        case LayoutKind::kCsr4:
            return run_multi<R, ApplyCSR<W, 4>>(nsys, hs, shifts, nshift, rhs, pvec, pidx, nproj, tol, G, info,
                                                use_graph, prec, &make_csr<W, 4>);
        case LayoutKind::kCsr16:
            return run_multi<R, ApplyCSR<W, 16>>(nsys, hs, shifts, nshift, rhs, pvec, pidx, nproj, tol, G, info,
                                                 use_graph, prec, &make_csr<W, 16>);
    }
    return SCOCG_ERR_INVALID;
}

}  // namespace
}  // namespace scocg

using namespace scocg;

extern "C" int scocg_solve_multi(int nsys, const scocg_handle* hs, const scocg_c128* const* shifts,
                                 const int* nshift, const void* const* rhs, const int64_t* const* proj_idx,
                                 const void* const* proj_vec, const int* nproj, double tol,
                                 scocg_c128* const* G_out, scocg_info* info, int use_graph) {
    if (nsys < 1 || nsys > 1024 || !hs || !shifts || !nshift || !rhs || !nproj || !G_out || !(tol >= 0.0) ||
        (proj_idx == nullptr) == (proj_vec == nullptr))
        return SCOCG_ERR_INVALID;
    const int prec = hs[0] ? hs[0]->opts.precision : -1;
    LayoutKind kind = LayoutKind::kBsr4;
    for (int s = 0; s < nsys; ++s) {
        scocg_ctx* h = hs[s];
        for (int t = 0; t < s; ++t)
            if (hs[t] == h) return SCOCG_ERR_INVALID;   // each system needs a workspace of its own
        if (!h || h->kind != HandleKind::kCsr || h->opts.precision != prec || h->stream != hs[0]->stream ||
            h->device != hs[0]->device || !shifts[s] || nshift[s] < 1 || nshift[s] > 4096 || !rhs[s] ||
            nproj[s] < 1 || nproj[s] > kMaxProj || !G_out[s] || (proj_vec && !proj_vec[s]) ||
            (proj_idx && !proj_idx[s]))
            return SCOCG_ERR_INVALID;
        const LayoutKind k = h->layout(false).kind;
        if (s == 0) kind = k;
        else if (k != kind) return SCOCG_ERR_INVALID;
        for (int k2 = 0; k2 < nshift[s]; ++k2)
            if (!std::isfinite(shifts[s][k2].re) || !std::isfinite(shifts[s][k2].im)) return SCOCG_ERR_INVALID;
        if (proj_idx)
            for (int m = 0; m < nproj[s]; ++m)
                if (proj_idx[s][m] < 0 || proj_idx[s][m] >= h->n) return SCOCG_ERR_INVALID;
    }
    if (prec == SCOCG_MIXED)
        return dispatch_layout<float>(kind, nsys, hs, shifts, nshift, rhs, proj_vec, proj_idx, nproj, tol, G_out,
                                      info, use_graph, prec);
    if (prec == SCOCG_MIXED_DF)
        return dispatch_layout<DF>(kind, nsys, hs, shifts, nshift, rhs, proj_vec, proj_idx, nproj, tol, G_out,
                                   info, use_graph, prec);
    return dispatch_layout<double>(kind, nsys, hs, shifts, nshift, rhs, proj_vec, proj_idx, nproj, tol, G_out, info,
                                   use_graph, prec);
}

extern "C" void scocg_multi_release(void) {
    if (g_plan) { g_plan->release(); delete g_plan; g_plan = nullptr; }
}

// A destroyed handle must not be reached through a cached plan.
void scocg::multi_forget(scocg_ctx* h) {
    if (!g_plan) return;
    for (scocg_ctx* p : g_plan->hs)
        if (p == h) { scocg_multi_release(); return; }
}
