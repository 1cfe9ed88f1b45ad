// Instantiations and launch of the persistent shifted-COCG kernel for every
// (precision, H layout) pair, plus a one-shot apply kernel y = (z - H) x.
#include <type_traits>

#include "solver_dispatch.cuh"

namespace scocg {

template <typename R, class Apply>
static int occupancy_of(size_t smem) {
    allow_dyn_smem<R, Apply>(smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, cocg_persistent<R, Apply>, kBlock, smem) != cudaSuccess)
        return 0;
    return nb;
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
    return a.resume ? launch_solve_resume<R>(a, h, grid, st) : launch_layout<R, false>(a, h, grid, st);
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
