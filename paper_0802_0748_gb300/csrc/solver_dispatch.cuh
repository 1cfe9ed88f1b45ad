// Launch of the persistent solve kernel for a CSR layout: the apply of each
// layout and vector precision, and the cooperative launch.  Included by
// solver.cu (solves from r_0 = b) and solver_resume.cu (continuations), so
// that the two sets of kernel instantiations compile in parallel.
#pragma once
#include <type_traits>

#include "solver_kernel.cuh"
#include "solver_launch.h"

namespace scocg {

// Dynamic shared memory above the 48 KB default (with the static part) needs
// the kernel's opt-in; the full-vector mode asks for up to kMaxFullShifts x
// kFullSmem bytes.
template <typename R, class Apply, bool kResume = false>
static void allow_dyn_smem(size_t smem) {
    if (smem > 0)
        cudaFuncSetAttribute((const void*)cocg_persistent<R, Apply, kResume>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename R, class Apply, bool kResume>
static cudaError_t coop_launch(const SolveArgs<R>& a, const Apply& ap, int grid, cudaStream_t st) {
    void* args[] = {(void*)&a, (void*)&ap};
    const size_t smem = a.Xf ? (size_t)a.K * kFullSmem : 0;
    allow_dyn_smem<R, Apply, kResume>(smem);
    return cudaLaunchCooperativeKernel((const void*)cocg_persistent<R, Apply, kResume>, dim3(grid), dim3(kBlock),
                                       args, smem, st);
}

// H values of each precision: FP64 for FP64 vectors, FP32 otherwise
template <typename W>
static const W* pick(const Layout& h, const double* d, const float* f);
template <> inline const double* pick<double>(const Layout&, const double* d, const float*) { return d; }
template <> inline const float* pick<float>(const Layout&, const double*, const float* f) { return f; }

// The blocked apply of vector precision R on layout h (row lanes on row-major
// blocks, or column lanes on the column-major copy for complex64 vectors).
template <typename R>
static typename BsrApply<R>::T make_bsr(const Layout& h, unsigned long long* dbg) {
    using W = typename ValT<R>::T;
    return typename BsrApply<R>::T{h.unit_off, h.bcol, pick<W>(h, h.bval64, h.bval32), h.n, h.nslots, dbg};
}
template <>
inline ApplyBSR4C<float> make_bsr<float>(const Layout& h, unsigned long long* dbg) {
    return ApplyBSR4C<float>{h.unit_off, h.bcol, h.bval32c, h.n, h.nslots, dbg};
}

template <typename R, bool kResume>
static cudaError_t launch_layout(const SolveArgs<R>& a, const Layout& h, int grid, cudaStream_t st) {
    using W = typename ValT<R>::T;
    switch (h.kind) {
        case LayoutKind::kBsr4: return coop_launch<R, typename BsrApply<R>::T, kResume>(a, make_bsr<R>(h, a.dbg), grid, st);
        case LayoutKind::kCsr1: {
            ApplyCSR<W, 1> ap{h.rowptr, h.col, pick<W>(h, h.val64, h.val32), h.n, h.nnz, a.dbg};
            return coop_launch<R, ApplyCSR<W, 1>, kResume>(a, ap, grid, st);
        }
        case LayoutKind::kCsr4: {
            ApplyCSR<W, 4> ap{h.rowptr, h.col, pick<W>(h, h.val64, h.val32), h.n, h.nnz, a.dbg};
            return coop_launch<R, ApplyCSR<W, 4>, kResume>(a, ap, grid, st);
        }
        case LayoutKind::kCsr16: {
            ApplyCSR<W, 16> ap{h.rowptr, h.col, pick<W>(h, h.val64, h.val32), h.n, h.nnz, a.dbg};
            return coop_launch<R, ApplyCSR<W, 16>, kResume>(a, ap, grid, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace scocg
