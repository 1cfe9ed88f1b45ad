// Density-matrix elements by the Fermi integral of Eq. densityM: one shifted
// COCG solve on a real-axis energy grid (broadened by delta) and a weighted
// reduction of Im G on the GPU.
#include <algorithm>
#include <cmath>
#include <vector>

#include "api_internal.h"

namespace scocg {
namespace {

// rho[j] = sum_k q[k] Im G[j][k], one warp per output, fixed summation order
__global__ void k_fermi_reduce(int nout, int K, const double2* G, const double* q, double* rho) {
    const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= nout) return;
    double s = 0.0;
    for (int k = lane; k < K; k += 32) s = fma(q[k], G[(size_t)j * K + k].y, s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rho[j] = s;
}

// Fermi-Dirac occupation f((e - mu) / kT); kT = 0 is the step function with
// f = 1/2 at e = mu.
double fermi(double e, double mu, double kT) {
    if (kT <= 0.0) return e < mu ? 1.0 : (e > mu ? 0.0 : 0.5);
    const double x = (e - mu) / kT;
    if (x > 0.0) { const double t = std::exp(-x); return t / (1.0 + t); }
    return 1.0 / (1.0 + std::exp(x));
}

}  // namespace
}  // namespace scocg

using namespace scocg;

extern "C" int scocg_density(scocg_handle h, double mu, double kT, double delta, double emin, double emax,
                             int nquad, const void* rhs, int nrhs, const int64_t* proj_idx, const void* proj_vec,
                             int nproj, double tol, double* rho_out, scocg_info* info) {
    if (!h || !rho_out || nquad < 2 || nquad > 4096 || !(delta > 0.0) || !(emax > emin) || !std::isfinite(mu) ||
        !(kT >= 0.0) || !std::isfinite(kT) || nrhs < 1 || nproj < 1)
        return SCOCG_ERR_INVALID;
    // grid, trapezoid weights and -1/pi f_k folded into one weight per shift
    std::vector<scocg_c128> z(nquad);
    std::vector<double> q(nquad);
    const double step = (emax - emin) / (nquad - 1);
    for (int k = 0; k < nquad; ++k) {
        const double e = emin + step * k;
        z[k].re = e;
        z[k].im = delta;
        const double w = (k == 0 || k == nquad - 1) ? 0.5 * step : step;
        q[k] = -w * fermi(e, mu, kT) / M_PI;
    }
    const size_t nout = (size_t)nrhs * nproj;
    double2* G = nullptr;
    double* d_q = nullptr;
    cudaError_t e = cudaMalloc(&G, sizeof(double2) * nout * nquad);
    if (e == cudaSuccess) e = cudaMalloc(&d_q, sizeof(double) * nquad);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_q, q.data(), sizeof(double) * nquad, cudaMemcpyHostToDevice, h->stream);
    int st = e == cudaSuccess ? SCOCG_OK : cuda_status(e);
    if (st == SCOCG_OK) {
        st = solve_impl(h, z.data(), nquad, rhs, nrhs, proj_idx, proj_vec, nproj, tol,
                        reinterpret_cast<scocg_c128*>(G), info, h->opts.precision, nullptr, nullptr);
        if (st >= 0) {
            const int threads = 256;
            const unsigned blocks = (unsigned)((nout * 32 + threads - 1) / threads);
            k_fermi_reduce<<<blocks, threads, 0, h->stream>>>((int)nout, nquad, G, d_q, rho_out);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) st = cuda_status(e);
        }
    }
    if (G) cudaFree(G);
    if (d_q) cudaFree(d_q);
    return st;
}
