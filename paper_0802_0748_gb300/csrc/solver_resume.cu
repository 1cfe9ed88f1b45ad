// The persistent solve kernels that continue a stopped solve (one per
// precision and CSR layout), compiled apart from the others.
#include "solver_dispatch.cuh"

namespace scocg {

template <typename R>
cudaError_t launch_solve_resume(const SolveArgs<R>& a, const Layout& h, int grid, cudaStream_t st) {
    return launch_layout<R, true>(a, h, grid, st);
}
template cudaError_t launch_solve_resume<double>(const SolveArgs<double>&, const Layout&, int, cudaStream_t);
template cudaError_t launch_solve_resume<float>(const SolveArgs<float>&, const Layout&, int, cudaStream_t);
template cudaError_t launch_solve_resume<DF>(const SolveArgs<DF>&, const Layout&, int, cudaStream_t);

}  // namespace scocg
