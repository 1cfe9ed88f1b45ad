// Hamiltonian set-up on the device: CSR validation (index range, sorted rows,
// exact symmetry H_ij == H_ji, FP32 representability, 4x4 block structure) and
// conversion of the caller's CSR into the solver's layouts (int32 CSR with
// FP64 and FP32 values; 4x4-blocked sliced ELL with FP64 and FP32 values).
#include "layout.h"

namespace scocg {

// ---------------------------------------------------------------- validation
__device__ __forceinline__ int64_t find_col(const int64_t* rowptr, const int32_t* col, int64_t row,
                                            int32_t c, bool sorted) {
    int64_t lo = rowptr[row], hi = rowptr[row + 1];
    if (sorted) {
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            const int32_t cm = col[mid];
            if (cm == c) return mid;
            if (cm < c) lo = mid + 1; else hi = mid;
        }
        return -1;
    }
    for (int64_t e = lo; e < hi; ++e)
        if (col[e] == c) return e;
    return -1;
}

// Pass 1: row pointers, column range, sortedness, FP32 representability.
__global__ void k_validate_rows(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                                const double* val, unsigned* flags) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned f = 0;
    const int64_t e0 = rowptr[i], e1 = rowptr[i + 1];
    if ((i == 0 && e0 != 0) || e1 < e0 || e1 > nnz || (i == n - 1 && e1 != nnz)) {
        atomicOr(flags, kFlagBadPtr);
        return;
    }
    int32_t prev = -1;
    for (int64_t e = e0; e < e1; ++e) {
        const int32_t c = col[e];
        if (c < 0 || c >= n) f |= kFlagBadCol;
        if (c <= prev) f |= kFlagUnsorted;
        prev = c;
        const double v = val[e];
        if (!isfinite(v)) f |= kFlagBadVal;
        if ((double)(float)v != v) f |= kFlagNotFp32;
    }
    if (f) atomicOr(flags, f);
}

// Pass 2 (only when pass 1 found valid indices): exact symmetry of every entry.
__global__ void k_validate_sym(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                               int sorted, unsigned* flags) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int32_t j = col[e];
        const int64_t t = find_col(rowptr, col, j, (int32_t)i, sorted != 0);
        if (t < 0 || val[t] != val[e]) { atomicOr(flags, kFlagUnsym); return; }
    }
}

// Pass 3: does the pattern consist of dense 4x4 blocks with the same block
// columns in each of the 4 rows of a block row?  (sorted rows, n % 4 == 0)
__global__ void k_check_bsr4(int64_t nbr, const int64_t* rowptr, const int32_t* col, unsigned* flags) {
    const int64_t B = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (B >= nbr) return;
    const int64_t r0 = 4 * B;
    const int64_t len = rowptr[r0 + 1] - rowptr[r0];
    if (len % 4) { atomicOr(flags, kFlagNotBsr4); return; }
    for (int r = 0; r < 4; ++r) {
        const int64_t e0 = rowptr[r0 + r];
        if (rowptr[r0 + r + 1] - e0 != len) { atomicOr(flags, kFlagNotBsr4); return; }
        for (int64_t t = 0; t < len; t += 4) {
            const int32_t c0 = col[e0 + t];
            if (c0 % 4 != 0 || c0 != col[rowptr[r0] + t]) { atomicOr(flags, kFlagNotBsr4); return; }
            for (int j = 1; j < 4; ++j)
                if (col[e0 + t + j] != c0 + j) { atomicOr(flags, kFlagNotBsr4); return; }
        }
    }
}

// ---------------------------------------------------------------- conversion
__global__ void k_to_csr32(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                           const double* val, int* rp32, int* col32, double* v64, float* v32) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i <= n) rp32[i] = (int)rowptr[i];
    if (i < nnz) {
        col32[i] = col[i];
        v64[i] = val[i];
        v32[i] = (float)val[i];
    }
}

// One thread per (block row, slot): slot t of block row B goes to
// unit u = B / 8, position br = B % 8, slot index unit_off[u] + t.
__global__ void k_to_bsr4(int64_t nbr, int64_t nunits, const int64_t* rowptr, const int32_t* col,
                          const double* val, const int* unit_off, int* bcol, double* bv64, float* bv32,
                          float* bv32c) {
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t u = tid / 8;
    if (u >= nunits) return;
    const int br = (int)(tid % 8);
    const int64_t B = u * 8 + br;
    const int s0 = unit_off[u], s1 = unit_off[u + 1];
    const int64_t nb = B < nbr ? (rowptr[4 * B + 1] - rowptr[4 * B]) / 4 : 0;
    for (int s = s0; s < s1; ++s) {
        const int64_t t = s - s0;
        const size_t slot = (size_t)s * 8 + br;
        if (t < nb) {
            bcol[slot] = col[rowptr[4 * B] + 4 * t] / 4;
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c) {
                    const double v = val[rowptr[4 * B + r] + 4 * t + c];
                    bv64[slot * 16 + r * 4 + c] = v;
                    bv32[slot * 16 + r * 4 + c] = (float)v;
                    bv32c[slot * 16 + c * 4 + r] = (float)v;
                }
        } else {
            bcol[slot] = -1;
            for (int e = 0; e < 16; ++e) { bv64[slot * 16 + e] = 0.0; bv32[slot * 16 + e] = 0.f; bv32c[slot * 16 + e] = 0.f; }
        }
    }
}

static inline unsigned grid1(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t validate_csr(int64_t n, int64_t nnz, const int64_t* d_rowptr, const int32_t* d_col,
                         const double* d_val, unsigned* d_flags, unsigned* h_flags, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_flags, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
    k_validate_rows<<<grid1(n, 256), 256, 0, st>>>(n, nnz, d_rowptr, d_col, d_val, d_flags);
    if ((e = cudaMemcpyAsync(h_flags, d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (*h_flags & (kFlagBadPtr | kFlagBadCol | kFlagBadVal)) return cudaSuccess;
    k_validate_sym<<<grid1(n, 256), 256, 0, st>>>(n, d_rowptr, d_col, d_val, (*h_flags & kFlagUnsorted) ? 0 : 1,
                                                  d_flags);
    if (!(*h_flags & kFlagUnsorted) && n % 4 == 0)
        k_check_bsr4<<<grid1(n / 4, 256), 256, 0, st>>>(n / 4, d_rowptr, d_col, d_flags);
    else
        k_check_bsr4<<<1, 1, 0, st>>>(0, d_rowptr, d_col, d_flags);
    if ((e = cudaMemcpyAsync(h_flags, d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if ((*h_flags & kFlagUnsorted) || n % 4 != 0) *h_flags |= kFlagNotBsr4;
    return cudaGetLastError();
}

cudaError_t convert_csr32(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col, const double* val,
                          int* rp32, int* col32, double* v64, float* v32, cudaStream_t st) {
    const int64_t m = nnz > n + 1 ? nnz : n + 1;
    k_to_csr32<<<grid1(m, 256), 256, 0, st>>>(n, nnz, rowptr, col, val, rp32, col32, v64, v32);
    return cudaGetLastError();
}

cudaError_t convert_bsr4(int64_t n, int64_t nunits, const int64_t* rowptr, const int32_t* col, const double* val,
                         const int* unit_off, int* bcol, double* bv64, float* bv32, float* bv32c, cudaStream_t st) {
    k_to_bsr4<<<grid1(nunits * 8, 256), 256, 0, st>>>(n / 4, nunits, rowptr, col, val, unit_off, bcol, bv64, bv32,
                                                      bv32c);
    return cudaGetLastError();
}

}  // namespace scocg
