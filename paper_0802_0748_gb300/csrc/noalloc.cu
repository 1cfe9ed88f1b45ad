// scocg_solve_csr_noalloc: the FP64 shifted-COCG solve for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at solve time: code running inside a
// memory pool or arena that owns all device memory, real-time loops that must
// not take the allocator's locks or risk fragmentation, and hosts that
// pre-reserve all memory up front.  This entry point needs no handle and makes
// no allocation: the caller passes H (device CSR, int32 row pointers), the
// shifts, b, the projections and the output G, and the solve's scratch (r, q,
// the per-shift state, the per-CTA partials and the control block) lives in one
// fixed file-scope device array, kScratchBytes long, that every GPU which loads
// this library holds until the process exits.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <cuda.h>   // driver types for the context id (entry points come through the runtime)

#include "api_internal.h"
#include "solver_kernel.cuh"

namespace scocg {

// Fixed scratch of the no-allocation solve.  Its size bounds the problems the
// entry point accepts (see scocg.h).
constexpr size_t kScratchBytes = size_t(24) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// The array's name in host code is only a host-side stand-in; its device
// address comes from cudaGetSymbolAddress, looked up with the device current.
// The address belongs to the module as loaded into one CUDA context: after
// cudaDeviceReset (or any teardown of the primary context) the module is
// loaded again and the array may move.  So the cache keeps, per device, the
// unique id of the context the address was taken in (cuCtxGetId through the
// runtime's driver entry points; no link against the driver library) and looks
// the symbol up again whenever the current context has another id.
constexpr int kMaxDevices = 64;
struct ScratchAddr {
    unsigned long long ctx_id;
    void* addr;
};
ScratchAddr g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mu;

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// Id of the calling thread's current context (0 when there is none yet).
cudaError_t current_ctx_id(unsigned long long* id) {
    static PfnCtxGetCurrent get_cur = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_cur || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorNotSupported;
        get_cur = reinterpret_cast<PfnCtxGetCurrent>(f1);
        get_id = reinterpret_cast<PfnCtxGetId>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_cur(&ctx) != CUDA_SUCCESS) return cudaErrorUnknown;
    *id = 0;
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorUnknown;
    return cudaSuccess;
}

// Device address of the scratch array in the current context of device `dev`
// (which must be current).  The first call in a context does the look-up.
cudaError_t scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long id = 0;
    cudaError_t e = current_ctx_id(&id);
    if (e != cudaSuccess) return e;
    if (id == 0 || g_scratch[dev].addr == nullptr || g_scratch[dev].ctx_id != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // creates the primary context if needed
        if (e != cudaSuccess) return e;
        e = current_ctx_id(&id);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = ScratchAddr{id, p};
    }
    *out = g_scratch[dev].addr;
    return cudaSuccess;
}

// A type of its own so that this file's kernel instantiations are distinct
// from the handle-based ones.
template <int LPR>
struct ApplyCSRFixed : ApplyCSR<double, LPR> {};

template <int LPR>
cudaError_t launch_csr(const SolveArgs<double>& a, const int* rowptr, const int* col, const double* val,
                       int64_t n, int64_t nnz, int grid, cudaStream_t st) {
    ApplyCSRFixed<LPR> ap{{rowptr, col, val, n, nnz, a.dbg}};
    void* args[] = {(void*)&a, (void*)&ap};
    return cudaLaunchCooperativeKernel((const void*)cocg_persistent<double, ApplyCSRFixed<LPR>>, dim3(grid),
                                       dim3(kBlock), args, 0, st);
}

template <int LPR>
int occupancy_csr() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cocg_persistent<double, ApplyCSRFixed<LPR>>, kBlock,
                                                      0) != cudaSuccess)
        return 0;
    return nb;
}

}  // namespace
}  // namespace scocg

using namespace scocg;

extern "C" int scocg_solve_csr_noalloc(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                                       const double* val, const scocg_c128* shifts, int nshift, const void* rhs,
                                       const int64_t* proj_idx, const void* proj_vec, int nproj, double tol,
                                       int max_iter, scocg_c128* G_out, scocg_info* info, void* cuda_stream) {
    if (n < 1 || nnz < 0 || !rowptr || (nnz > 0 && (!col || !val)) || !shifts || nshift < 1 || nshift > 4096 ||
        !rhs ||
        nproj < 1 || nproj > kMaxProj || (proj_idx == nullptr) == (proj_vec == nullptr) || !G_out || !(tol >= 0.0))
        return SCOCG_ERR_INVALID;
    for (int k = 0; k < nshift; ++k)
        if (!std::isfinite(shifts[k].re) || !std::isfinite(shifts[k].im)) return SCOCG_ERR_INVALID;
    if (proj_idx)
        for (int m = 0; m < nproj; ++m)
            if (proj_idx[m] < 0 || proj_idx[m] >= n) return SCOCG_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e);

    const double avg = (double)nnz / (double)n;
    const int lpr = avg <= 4.0 ? 1 : (avg <= 24.0 ? 4 : 16);
    const int occ = lpr == 1 ? occupancy_csr<1>() : (lpr == 4 ? occupancy_csr<4>() : occupancy_csr<16>());
    if (occ <= 0) return SCOCG_ERR_CUDA;
    const int rpu = 32 / lpr;
    const int64_t nunits = (n + rpu - 1) / rpu;
    const int K = nshift, M = nproj;
    int64_t want = std::max<int64_t>((nunits + kWarps - 1) / kWarps, (K + kBlock - 1) / kBlock);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)occ * sms));
    if ((int64_t)grid * kBlock < K) return SCOCG_ERR_TOO_LARGE;
    const int strideB = 3 + 2 * M + 1;

    // carve the fixed scratch (measure first: sizes beyond it are refused)
    void* base = nullptr;
    SolveArgs<double> a{};
    Ctrl* ctrl = nullptr;
    auto carve = [&](Carver& c) {
        ctrl = (Ctrl*)c.take(sizeof(Ctrl));
        a.r = (double2*)c.take(sizeof(double2) * (size_t)n);
        a.q = (double2*)c.take(sizeof(double2) * (size_t)n);
        a.cidx = proj_idx ? (const int64_t*)c.take(sizeof(int64_t) * M) : nullptr;
        a.z = (const double2*)c.take(sizeof(double2) * K);
        a.S.pi_prev = (double2*)c.take(sizeof(double2) * K);
        a.S.pi_cur = (double2*)c.take(sizeof(double2) * K);
        a.S.sigma = (double2*)c.take(sizeof(double2) * K);
        a.S.alpha_k = (double2*)c.take(sizeof(double2) * K);
        a.S.inv_cur = (double2*)c.take(sizeof(double2) * K);
        a.S.P = (double2*)c.take(sizeof(double2) * (size_t)K * M);
        a.S.X = (double2*)c.take(sizeof(double2) * (size_t)K * M);
        a.S.frozen = (int*)c.take(sizeof(int) * K);
        a.S.iters = (int*)c.take(sizeof(int) * K);
        a.S.resid = (double*)c.take(sizeof(double) * K);
        a.partA = (double*)c.take(sizeof(double) * grid * 4);
        a.partB = (double*)c.take(sizeof(double) * grid * strideB);
        a.partC = (double*)c.take(sizeof(double) * grid * kPartC);
    };
    Carver measure{nullptr, 0};
    carve(measure);
    if (measure.off > kScratchBytes) return SCOCG_ERR_TOO_LARGE;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess) return cuda_status(e);
    Carver cut{static_cast<char*>(base), 0};
    carve(cut);

    // the control block (barrier counter, status, statistics) must start at
    // zero; everything else is written by the kernel before it is read
    e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void*)a.z, shifts, sizeof(double2) * K, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && proj_idx)
        e = cudaMemcpyAsync((void*)a.cidx, proj_idx, sizeof(int64_t) * M, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e);

    scocg_opts o;
    fill_opts(o, nullptr);
    a.n = n;
    a.nunits = nunits;
    a.rows_per_unit = rpu;
    a.b = static_cast<const double2*>(rhs);
    a.cvec = static_cast<const double2*>(proj_vec);
    a.nproj = M;
    a.K = K;
    a.seed = default_seed(shifts, K);   // the rule scocg_solve uses (host memory only)
    a.allow_switch = 1;
    a.tol = tol;
    a.max_iter = max_iter > 0 ? max_iter : o.max_iter;
    a.strideB = strideB;
    a.sync.count = &ctrl->count;
    a.sync.status = &ctrl->status;
    a.sync.timeout_ns = (uint64_t)(o.timeout_ms * 1e6);
    a.sync.nctas = grid;
    a.stats = &ctrl->stats;
    a.G = reinterpret_cast<double2*>(G_out);
    a.dbg = ctrl->dbg;

    e = lpr == 1 ? launch_csr<1>(a, rowptr, col, val, n, nnz, grid, st)
      : lpr == 4 ? launch_csr<4>(a, rowptr, col, val, n, nnz, grid, st)
                 : launch_csr<16>(a, rowptr, col, val, n, nnz, grid, st);
    Ctrl c;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && info && info->freeze_iter)
        e = cudaMemcpyAsync(info->freeze_iter, a.S.iters, sizeof(int) * K, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && info && info->resid)
        e = cudaMemcpyAsync(info->resid, a.S.resid, sizeof(double) * K, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    // checked builds: an out-of-range row pointer or column index of the
    // caller's CSR was recorded (and skipped) by the kernel
    if (c.dbg[0]) return SCOCG_ERR_INVALID;
    if (info) {
        if (info->resid)   // the kernel keeps squared residual estimates
            for (int k = 0; k < K; ++k) info->resid[k] = std::sqrt(info->resid[k]);
        info->iters = c.stats.iters;
        info->n_switch = c.stats.n_switch;
        info->seed_final = c.stats.seed;
        info->n_replace = 0;
        info->shift_iters = c.stats.shift_iters;
        info->seconds = 0.0;
        info->bytes_per_iter = (double)nnz * 12.0 + 4.0 * (n + 1) + (6.0 + (proj_vec ? M : 0)) * 16.0 * n;
    }
    return c.status < 0 ? c.status : c.stats.status;
}
