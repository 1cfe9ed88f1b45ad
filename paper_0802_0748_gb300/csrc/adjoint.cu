// Full-vector shifted COCG and the adjoint gradient (placeholder until built).
#include "api_internal.h"

namespace scocg {

int solve_full_impl(scocg_ctx* h, const scocg_c128* shifts, int nshift, const void* rhs, double tol, void* X_out,
                    scocg_info* info) {
    (void)h; (void)shifts; (void)nshift; (void)rhs; (void)tol; (void)X_out; (void)info;
    return SCOCG_ERR_INVALID;
}

int grad_impl(scocg_ctx* h, const scocg_c128* shifts, int nshift, const void* rhs, int nrhs,
              const int64_t* proj_idx, const void* proj_vec, int nproj, double tol, const scocg_c128* dL_dG,
              double* dL_dval, scocg_info* info) {
    (void)h; (void)shifts; (void)nshift; (void)rhs; (void)nrhs; (void)proj_idx; (void)proj_vec; (void)nproj;
    (void)tol; (void)dL_dG; (void)dL_dval; (void)info;
    return SCOCG_ERR_INVALID;
}

}  // namespace scocg
