// Full-vector shifted COCG and the adjoint gradient of a real loss L(G)
// with respect to the stored CSR values.
//
// With A_k = z_k I - H, x_k = A_k^{-1} b and y_mk = A_k^{-1} c_m (A_k is
// complex symmetric, so the adjoint system is a forward solve with c_m as the
// right-hand side), dG_mk / dH_ab = y_mk[a] x_k[b], and for dL/dG given in the
// convention dL/dRe G + i dL/dIm G:
//   dL/dH_ab = Re sum_{k,m} conj(dL/dG_mk) y_mk[a] x_k[b]
// evaluated on every stored entry (a, b) (a sampled dense-dense product over
// the CSR pattern).  Shifts are processed in chunks whose [chunk][N] vectors
// fit the memory budget; each chunk re-solves (vectors are recomputed, not
// kept).
#include <algorithm>
#include <cmath>
#include <vector>

#include "api_internal.h"

namespace scocg {

// y^T[n][kc] = x[kc][n] (complex128), tiled through shared memory
__global__ void k_transpose(int64_t n, int kc, const double2* x, double2* y) {
    __shared__ double2 tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int k = k0 + r;
        const int64_t i = i0 + tx;
        if (k < kc && i < n) tile[r][tx] = x[(size_t)k * n + i];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + r;
        const int k = k0 + tx;
        if (k < kc && i < n) y[(size_t)i * kc + k] = tile[tx][r];
    }
}

// One warp per CSR row a: ybar_k = conj(gbar_k) y_k[a] in registers (lanes
// over shifts), then for each stored (a, b): g += Re sum_k ybar_k x_k[b] with
// x read shift-contiguous from xT[b][kc].
__global__ void k_sddmm_grad(int64_t n, int kc, const int* rowptr, const int* col, const double2* xT,
                             const double2* y, const double2* gbar, double* grad) {
    const int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (a >= n) return;
    constexpr int kPer = kMaxFullShifts / 32;
    double2 yb[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        const int k = lane + 32 * j;
        if (k < kc) {
            const double2 g = gbar[k];
            const double2 yk = y[(size_t)k * n + a];
            yb[j] = cmul(c2(g.x, -g.y), yk);
        } else {
            yb[j] = c2(0, 0);
        }
    }
    for (int e = rowptr[a]; e < rowptr[a + 1]; ++e) {
        const double2* xb = xT + (size_t)col[e] * kc;
        double sre = 0.0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int k = lane + 32 * j;
            if (k < kc) {
                const double2 xv = xb[k];
                sre = fma(yb[j].x, xv.x, fma(-yb[j].y, xv.y, sre));
            }
        }
        sre = warp_sum(sre);
        if (lane == 0) grad[e] += sre;
    }
}

// flag = 1 unless v equals the unit vector e_j (v device complex128 [n])
__global__ void k_differs_from_unit(int64_t n, const double2* v, int64_t j, int* flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 w = v[i];
        const double ex = i == j ? 1.0 : 0.0;
        if (w.x != ex || w.y != 0.0) atomicOr(flag, 1);
    }
}
__global__ void k_differs(int64_t n, const double2* u, const double2* v, int* flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = u[i], b = v[i];
        if (a.x != b.x || a.y != b.y) atomicOr(flag, 1);
    }
}
__global__ void k_unit(int64_t n, int64_t j, double2* v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = c2(i == j ? 1.0 : 0.0, 0.0);
}

int solve_full_impl(scocg_ctx* h, const scocg_c128* shifts, int nshift, const void* rhs, double tol, void* X_out,
                    scocg_info* info) {
    if (!h || !shifts || nshift < 1 || !rhs || !X_out) return SCOCG_ERR_INVALID;
    const int64_t n = h->n;
    // per chunk: p vectors in a workspace of their own, the G of the dummy projection
    const int chunk = std::min(nshift, kMaxFullShifts);
    double2* P = nullptr;
    scocg_c128* G = nullptr;
    cudaError_t e = cudaMalloc(&P, sizeof(double2) * (size_t)chunk * n);
    if (e == cudaSuccess) e = cudaMalloc(&G, sizeof(scocg_c128) * chunk);
    if (e != cudaSuccess) { cudaFree(P); cudaFree(G); return cuda_status(e); }
    int worst = SCOCG_OK;
    scocg_info acc{};
    std::vector<int> fi;
    std::vector<double> rs;
    for (int k0 = 0; k0 < nshift && worst >= 0; k0 += chunk) {
        const int kc = std::min(chunk, nshift - k0);
        scocg_info ci{};
        fi.assign(kc, 0); rs.assign(kc, 0.0);
        ci.freeze_iter = fi.data();
        ci.resid = rs.data();
        const int64_t idx0 = 0;
        double2* X = static_cast<double2*>(X_out) + (size_t)k0 * n;
        int st = solve_impl(h, shifts + k0, kc, rhs, 1, &idx0, nullptr, 1, tol, G, &ci, SCOCG_FP64, X, P);
        if (st < 0) { worst = st; break; }
        if (st == SCOCG_NOT_CONVERGED) worst = SCOCG_NOT_CONVERGED;
        acc.iters = std::max(acc.iters, ci.iters);
        acc.n_switch += ci.n_switch;
        acc.shift_iters += ci.shift_iters;
        acc.seconds += ci.seconds;
        acc.seed_final = ci.seed_final;
        acc.bytes_per_iter = ci.bytes_per_iter + 4.0 * 16.0 * (double)kc * (double)n;
        if (info) {
            if (info->freeze_iter) std::copy(fi.begin(), fi.end(), info->freeze_iter + k0);
            if (info->resid) std::copy(rs.begin(), rs.end(), info->resid + k0);
        }
    }
    cudaFree(P);
    cudaFree(G);
    if (info) {
        int* f = info->freeze_iter;
        double* r = info->resid;
        *info = acc;
        info->freeze_iter = f;
        info->resid = r;
    }
    return worst;
}

int grad_impl(scocg_ctx* h, const scocg_c128* shifts, int nshift, const void* rhs, int nrhs,
              const int64_t* proj_idx, const void* proj_vec, int nproj, double tol, const scocg_c128* dL_dG,
              double* dL_dval, scocg_info* info) {
    if (!h || h->kind != HandleKind::kCsr || !shifts || nshift < 1 || !rhs || nrhs != 1 || nproj < 1 ||
        nproj > kMaxProj || (proj_idx == nullptr) == (proj_vec == nullptr) || !dL_dG || !dL_dval || !(tol >= 0.0))
        return SCOCG_ERR_INVALID;
    const int64_t n = h->n, nnz = h->nnz;
    if (proj_idx)
        for (int m = 0; m < nproj; ++m)
            if (proj_idx[m] < 0 || proj_idx[m] >= n) return SCOCG_ERR_INVALID;
    cudaStream_t s = h->stream;
    // chunk so that x, y, the transpose and p ([chunk][n] complex128 each) fit
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const size_t per_shift = 4 * sizeof(double2) * (size_t)n;
    int chunk = (int)std::min<size_t>((size_t)std::min(nshift, kMaxFullShifts), std::max<size_t>(1, free_b / 2 / per_shift));
    double2 *X = nullptr, *Y = nullptr, *XT = nullptr, *C = nullptr, *gb = nullptr;
    int* d_flag = nullptr;
    cudaError_t e = cudaMalloc(&X, sizeof(double2) * (size_t)chunk * n);
    if (e == cudaSuccess) e = cudaMalloc(&Y, sizeof(double2) * (size_t)chunk * n);
    if (e == cudaSuccess) e = cudaMalloc(&XT, sizeof(double2) * (size_t)chunk * n);
    if (e == cudaSuccess) e = cudaMalloc(&C, sizeof(double2) * n);
    if (e == cudaSuccess) e = cudaMalloc(&gb, sizeof(double2) * chunk);
    if (e == cudaSuccess) e = cudaMalloc(&d_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(dL_dval, 0, sizeof(double) * std::max<int64_t>(nnz, 1), s);
    int worst = SCOCG_OK;
    if (e != cudaSuccess) worst = cuda_status(e);
    scocg_info acc{};
    // does c_m equal b?  (then y_mk = x_k and the adjoint solve is the forward one)
    std::vector<int> same(nproj, 0);
    for (int m = 0; m < nproj && worst >= 0; ++m) {
        int flag = 0;
        e = cudaMemsetAsync(d_flag, 0, sizeof(int), s);
        if (e == cudaSuccess) {
            if (proj_idx) k_differs_from_unit<<<256, 256, 0, s>>>(n, (const double2*)rhs, proj_idx[m], d_flag);
            else k_differs<<<256, 256, 0, s>>>(n, (const double2*)rhs, (const double2*)proj_vec + (size_t)m * n, d_flag);
            e = cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { worst = cuda_status(e); break; }
        same[m] = !flag;
    }
    for (int k0 = 0; k0 < nshift && worst >= 0; k0 += chunk) {
        const int kc = std::min(chunk, nshift - k0);
        scocg_info ci{};
        int st = solve_full_impl(h, shifts + k0, kc, rhs, tol, X, &ci);
        if (st < 0) { worst = st; break; }
        if (st == SCOCG_NOT_CONVERGED) worst = SCOCG_NOT_CONVERGED;
        acc.iters = std::max(acc.iters, ci.iters); acc.shift_iters += ci.shift_iters; acc.seconds += ci.seconds;
        acc.n_switch += ci.n_switch;
        dim3 tb(32, 8), tg((unsigned)((n + 31) / 32), (unsigned)((kc + 31) / 32));
        k_transpose<<<tg, tb, 0, s>>>(n, kc, X, XT);
        for (int m = 0; m < nproj && worst >= 0; ++m) {
            const double2* Ym = X;
            if (!same[m]) {
                const double2* cm;
                if (proj_idx) { k_unit<<<256, 256, 0, s>>>(n, proj_idx[m], C); cm = C; }
                else cm = (const double2*)proj_vec + (size_t)m * n;
                scocg_info cy{};
                st = solve_full_impl(h, shifts + k0, kc, cm, tol, Y, &cy);
                if (st < 0) { worst = st; break; }
                if (st == SCOCG_NOT_CONVERGED) worst = SCOCG_NOT_CONVERGED;
                acc.shift_iters += cy.shift_iters; acc.seconds += cy.seconds;
                Ym = Y;
            }
            e = cudaMemcpyAsync(gb, (const double2*)dL_dG + (size_t)m * nshift + k0, sizeof(double2) * kc,
                                cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) { worst = cuda_status(e); break; }
            const int64_t threads = n * 32;
            k_sddmm_grad<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(n, kc, h->d_rowptr, h->d_col, XT, Ym, gb,
                                                                           dL_dval);
            e = cudaGetLastError();
            if (e != cudaSuccess) { worst = cuda_status(e); break; }
        }
    }
    if (worst >= 0) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) worst = cuda_status(e);
    }
    cudaFree(X); cudaFree(Y); cudaFree(XT); cudaFree(C); cudaFree(gb); cudaFree(d_flag);
    if (info) {
        info->iters = acc.iters; info->n_switch = acc.n_switch; info->shift_iters = acc.shift_iters;
        info->seconds = acc.seconds; info->seed_final = acc.seed_final;
    }
    return worst;
}

}  // namespace scocg
