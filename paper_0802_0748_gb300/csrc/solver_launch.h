// Host-side interface between the C ABI and the solver kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "solver.cuh"

namespace scocg {

enum class LayoutKind : int { kBsr4 = 0, kCsr1 = 1, kCsr4 = 2, kCsr16 = 3 };

// Device layout of a CSR Hamiltonian (owned by the handle).
struct Layout {
    LayoutKind kind;
    int64_t n;
    int64_t nnz;
    // int32 CSR (always present)
    const int* rowptr;
    const int* col;
    const double* val64;
    const float* val32;
    // 4x4-blocked sliced ELL (kind == kBsr4)
    int64_t nunits_bsr;
    int64_t nslots;
    const int* unit_off;
    const int* bcol;
    const double* bval64;
    const float* bval32;     // blocks row-major
    const float* bval32c;    // the same blocks column-major (complex64 applies)
};

int rows_per_unit(LayoutKind k);
int max_coresident_ctas(const Layout& h, int precision, int num_sms, size_t dyn_smem = 0);

template <typename R>
cudaError_t launch_solve(const SolveArgs<R>& a, const Layout& h, int grid, cudaStream_t st);
// the continuation kernels (a.resume = 1), compiled in solver_resume.cu
template <typename R>
cudaError_t launch_solve_resume(const SolveArgs<R>& a, const Layout& h, int grid, cudaStream_t st);

cudaError_t launch_apply(const Layout& h, int precision, double2 z, const void* x, void* y, cudaStream_t st);

}  // namespace scocg
