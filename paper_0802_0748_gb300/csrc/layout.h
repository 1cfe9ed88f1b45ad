// Host-callable set-up routines for the Hamiltonian layouts (see layout.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace scocg {

enum : unsigned {
    kFlagBadPtr = 1u,      // rowptr not monotone / wrong ends
    kFlagBadCol = 2u,      // column index out of range
    kFlagUnsym = 4u,       // some H_ij != H_ji (or (j,i) missing)
    kFlagUnsorted = 8u,    // a row's columns are not strictly increasing
    kFlagNotFp32 = 16u,    // some value is not exactly representable in FP32
    kFlagNotBsr4 = 32u,    // pattern is not made of dense 4x4 blocks
    kFlagBadVal = 64u,     // non-finite value
};

cudaError_t validate_csr(int64_t n, int64_t nnz, const int64_t* d_rowptr, const int32_t* d_col,
                         const double* d_val, unsigned* d_flags, unsigned* h_flags, cudaStream_t st);
cudaError_t convert_csr32(int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col, const double* val,
                          int* rp32, int* col32, double* v64, float* v32, cudaStream_t st);
cudaError_t convert_bsr4(int64_t n, int64_t nunits, const int64_t* rowptr, const int32_t* col, const double* val,
                         const int* unit_off, int* bcol, double* bv64, float* bv32, float* bv32c,
                         cudaStream_t st);

}  // namespace scocg
