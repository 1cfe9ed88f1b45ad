// Instantiations and launch of the persistent shifted-COCG kernel for every
// (precision, H layout) pair, plus a one-shot apply kernel y = (z - H) x.
#include <type_traits>

#include "solver_kernel.cuh"
#include "solver_launch.h"

namespace scocg {

// Dynamic shared memory above the 48 KB default (with the static part) needs
// the kernel's opt-in; the full-vector mode asks for up to kMaxFullShifts x
// kFullSmem bytes.
template <typename R, class Apply>
static void allow_dyn_smem(size_t smem) {
    if (smem > 0)
        cudaFuncSetAttribute((const void*)cocg_persistent<R, Apply>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
}

template <typename R, class Apply>
static cudaError_t coop_launch(const SolveArgs<R>& a, const Apply& ap, int grid, cudaStream_t st) {
    void* args[] = {(void*)&a, (void*)&ap};
    const size_t smem = a.Xf ? (size_t)a.K * kFullSmem : 0;
    allow_dyn_smem<R, Apply>(smem);
    return cudaLaunchCooperativeKernel((const void*)cocg_persistent<R, Apply>, dim3(grid), dim3(kBlock), args, smem,
                                       st);
}

template <typename R, class Apply>
static int occupancy_of(size_t smem) {
    allow_dyn_smem<R, Apply>(smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cocg_persistent<R, Apply>, kBlock, smem) != cudaSuccess)
        return 0;
    return nb;
}

// H values of each precision: FP64 for FP64 vectors, FP32 otherwise
template <typename W>
static const W* pick(const Layout& h, const double* d, const float* f);
template <> const double* pick<double>(const Layout&, const double* d, const float*) { return d; }
template <> const float* pick<float>(const Layout&, const double*, const float* f) { return f; }

// The blocked apply of vector precision R on layout h (row lanes on row-major
// blocks, or column lanes on the column-major copy for complex64 vectors).
template <typename R>
static typename BsrApply<R>::T make_bsr(const Layout& h, unsigned long long* dbg) {
    using W = typename ValT<R>::T;
    return typename BsrApply<R>::T{h.unit_off, h.bcol, pick<W>(h, h.bval64, h.bval32), h.n, h.nslots, dbg};
}
template <>
ApplyBSR4C<float> make_bsr<float>(const Layout& h, unsigned long long* dbg) {
    return ApplyBSR4C<float>{h.unit_off, h.bcol, h.bval32c, h.n, h.nslots, dbg};
}

template <typename R>
static int dispatch_occ(const Layout& h, size_t smem) {
    using W = typename ValT<R>::T;
    switch (h.kind) {
        case LayoutKind::kBsr4: return occupancy_of<R, typename BsrApply<R>::T>(smem);
        case LayoutKind::kCsr1: return occupancy_of<R, ApplyCSR<W, 1>>(smem);
        case LayoutKind::kCsr4: return occupancy_of<R, ApplyCSR<W, 4>>(smem);
        case LayoutKind::kCsr16: return occupancy_of<R, ApplyCSR<W, 16>>(smem);
    }
    return 0;
}

int max_coresident_ctas(const Layout& h, int precision, int num_sms, size_t dyn_smem) {
    const int occ = precision == SCOCG_MIXED ? dispatch_occ<float>(h, dyn_smem)
                  : precision == SCOCG_MIXED_DF ? dispatch_occ<DF>(h, dyn_smem) : dispatch_occ<double>(h, dyn_smem);
    return occ * num_sms;
}

int rows_per_unit(LayoutKind k) {
    switch (k) {
        case LayoutKind::kBsr4: return 32;
        case LayoutKind::kCsr1: return 32;
        case LayoutKind::kCsr4: return 8;
        case LayoutKind::kCsr16: return 2;
    }
    return 32;
}

template <typename R>
cudaError_t launch_solve(const SolveArgs<R>& a, const Layout& h, int grid, cudaStream_t st) {
    using W = typename ValT<R>::T;
    switch (h.kind) {
        case LayoutKind::kBsr4: return coop_launch(a, make_bsr<R>(h, a.dbg), grid, st);
        case LayoutKind::kCsr1: {
            ApplyCSR<W, 1> ap{h.rowptr, h.col, pick<W>(h, h.val64, h.val32), h.n, h.nnz, a.dbg};
            return coop_launch(a, ap, grid, st);
        }
        case LayoutKind::kCsr4: {
            ApplyCSR<W, 4> ap{h.rowptr, h.col, pick<W>(h, h.val64, h.val32), h.n, h.nnz, a.dbg};
            return coop_launch(a, ap, grid, st);
        }
        case LayoutKind::kCsr16: {
            ApplyCSR<W, 16> ap{h.rowptr, h.col, pick<W>(h, h.val64, h.val32), h.n, h.nnz, a.dbg};
            return coop_launch(a, ap, grid, st);
        }
    }
    return cudaErrorInvalidValue;
}
template cudaError_t launch_solve<double>(const SolveArgs<double>&, const Layout&, int, cudaStream_t);
template cudaError_t launch_solve<float>(const SolveArgs<float>&, const Layout&, int, cudaStream_t);
template cudaError_t launch_solve<DF>(const SolveArgs<DF>&, const Layout&, int, cudaStream_t);

// ---------------------------------------------------------------- one apply
template <typename R, typename VV, class Apply>
__global__ void __launch_bounds__(256) k_apply(Apply ap, int64_t nunits, VV zs, const VV* x, VV* y) {
    const int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (u >= nunits) return;
    int64_t row;
    VV w;
    if (ap(u, lane, zs, x, row, w)) y[row] = w;
}

template <typename R, typename VV, class Apply>
static cudaError_t apply_one(const Apply& ap, int64_t nunits, VV zs, const VV* x, VV* y, cudaStream_t st) {
    const int64_t threads = nunits * 32;
    k_apply<R, VV, Apply><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(ap, nunits, zs, x, y);
    return cudaGetLastError();
}

template <typename R, typename VV>
static cudaError_t apply_dispatch(const Layout& h, int64_t nunits, VV zs, const VV* x, VV* y, cudaStream_t st) {
    switch (h.kind) {
        case LayoutKind::kBsr4:
            if constexpr (std::is_same<VV, float2>::value)   // complex64: column lanes
                return apply_one<R, VV>(make_bsr<float>(h, nullptr), nunits, zs, x, y, st);
            else
                return apply_one<R, VV>(ApplyBSR4<R>{h.unit_off, h.bcol, pick<R>(h, h.bval64, h.bval32), h.n, h.nslots, nullptr}, nunits, zs, x, y, st);
        case LayoutKind::kCsr1:
            return apply_one<R, VV>(ApplyCSR<R, 1>{h.rowptr, h.col, pick<R>(h, h.val64, h.val32), h.n, h.nnz, nullptr}, nunits, zs, x, y, st);
        case LayoutKind::kCsr4:
            return apply_one<R, VV>(ApplyCSR<R, 4>{h.rowptr, h.col, pick<R>(h, h.val64, h.val32), h.n, h.nnz, nullptr}, nunits, zs, x, y, st);
        case LayoutKind::kCsr16:
            return apply_one<R, VV>(ApplyCSR<R, 16>{h.rowptr, h.col, pick<R>(h, h.val64, h.val32), h.n, h.nnz, nullptr}, nunits, zs, x, y, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_apply(const Layout& h, int precision, double2 z, const void* x, void* y, cudaStream_t st) {
    const int64_t nunits = (h.n + rows_per_unit(h.kind) - 1) / rows_per_unit(h.kind);
    if (precision == SCOCG_MIXED)
        return apply_dispatch<float, float2>(h, nunits, make_float2((float)z.x, (float)z.y), (const float2*)x,
                                             (float2*)y, st);
    if (precision == SCOCG_MIXED_DF)
        return apply_dispatch<float, float4>(h, nunits, df_from(z), (const float4*)x, (float4*)y, st);
    return apply_dispatch<double, double2>(h, nunits, z, (const double2*)x, (double2*)y, st);
}

}  // namespace scocg
