// Handle structure and internal entry points shared by the C-ABI translation units.
#pragma once
#include <vector>
#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"
#include "solver_launch.h"

namespace scocg {

enum class HandleKind : int { kCsr = 0, kHubbard = 1 };

// Device control block of one solve: barrier counter, status word, statistics.
struct Ctrl {
    unsigned long long count;
    int status;
    int pad;
    SolveStats stats;
    unsigned long long dbg[4];   // checked builds: (flag, site, index, limit)
};

// Sequential carving of a buffer into 256-byte aligned pieces; with a null
// base it only measures (every piece returns nullptr, `off` is the total).
struct Carver {
    char* base;
    size_t off;
    void* take(size_t bytes) {
        void* p = base ? base + off : nullptr;
        off += ((bytes + 255) / 256) * 256;
        return p;
    }
};

// Grow-only device workspace carved into 256-byte aligned pieces.
struct Workspace {
    void* base = nullptr;
    size_t cap = 0;
    size_t off = 0;
    unsigned long long* gen = nullptr;   // bumped on every (re)allocation
    cudaError_t reserve(size_t bytes);   // resets the carve offset
    // the same, keeping the first `keep` bytes when the buffer has to grow
    cudaError_t reserve_keep(size_t bytes, size_t keep, cudaStream_t s);
    void* get(size_t bytes);
    void release();
};

// Matrix-free extended Hubbard model (per-spin tables built on the device).
struct Hubbard {
    int L = 0, n_up = 0, n_dn = 0, periodic = 0;
    double t = 0, U = 0, V = 0;
    int D_up = 0, D_dn = 0;
    int64_t nunits = 0;
    // tables for spin s at offset s * (table stride) in each array
    uint32_t* d_states = nullptr;   // [2][Dmax]
    int32_t* d_hop_target = nullptr;   // [2][Dmax][2L]
    int8_t* d_hop_sign = nullptr;      // [2][Dmax][2L]
    int32_t* d_hop_packed = nullptr;   // [2][Dmax][2L]: (target << 1) | (sign < 0), -1 = unused
    float2* d_diagf = nullptr;         // [(L+1)(4L+1)]: U cu + V cv as float pairs (hi, lo)
    int Dmax = 0;
    double table_bytes = 0;
    // model 1: two orbitals per site on a cluster (L = 2 ns modes per spin;
    // t, U, V above unused).  Tables per spin at offset spin * (table stride).
    int model = 0;                     // 0: one-orbital ring, 1: two-orbital cluster
    int ns = 0, nb = 0, S2 = 0;        // sites, bonds, hop slots per rank
    double Up = 0, J = 0, Jp = 0;
    int32_t* d_hop2 = nullptr;         // [2][Dmax][S2]: (target << 8) | (amplitude << 1) | (sign < 0), -1 = unused
    int32_t* d_orb2 = nullptr;         // [2][Dmax][ns]: (target << 1) | destination orbital, -1 = no move
    uint32_t* d_nib2 = nullptr;        // [2][Dmax][2]: site occupations n_i and (A n)_i as nibbles
    double* d_self2 = nullptr;         // [2][Dmax]: the diagonal terms of one spin alone
    float2* d_self2f = nullptr;        // [2][Dmax]: the same as float pairs (hi, lo)
    double* d_amp2 = nullptr;          // [nb][2][2] hoppings t_ab of each bond
    float2* d_amp2f = nullptr;         // [nb][2][2][2] the same with each sign, as (hi, hi, lo, lo) float4s
    double* d_cross2 = nullptr;        // [3][kCross2]: U c, U' c, V c for small integer counts c
    float2* d_cross2f = nullptr;       // the same as float pairs
    int32_t* d_bonds2 = nullptr;       // [nb][2]
};

}  // namespace scocg

namespace scocg {
// One autotuner decision for block (multi-right-hand-side) solves.
struct TuneEntry {
    int prec, K, M, nrhs;   // key: precision, shifts, projections, min(nrhs, 32)
    int T, per_sm;          // slots per launch, CTAs per SM (0 = occupancy maximum)
};
}  // namespace scocg

struct scocg_ctx {
    scocg::HandleKind kind = scocg::HandleKind::kCsr;
    int64_t n = 0, nnz = 0;
    scocg_opts opts{};
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    // CSR layouts
    int* d_rowptr = nullptr;
    int* d_col = nullptr;
    double* d_val64 = nullptr;
    float* d_val32 = nullptr;
    bool bsr_ok = false;
    bool fp32_exact = false;
    int64_t nunits_bsr = 0, nslots = 0;
    int* d_unit_off = nullptr;
    int* d_bcol = nullptr;
    double* d_bval64 = nullptr;
    float* d_bval32 = nullptr;
    float* d_bval32c = nullptr;      // the FP32 blocks column-major
    scocg::LayoutKind csr_kind = scocg::LayoutKind::kCsr1;
    int force_kind = -1;       // tuning override of the CSR lanes-per-row layout
    // Hubbard
    scocg::Hubbard hub;
    // per-solve state
    scocg::Ctrl* d_ctrl = nullptr;
    scocg::Workspace ws;
    unsigned long long ws_gen = 0;   // changes whenever ws is (re)allocated or the handle is new
    std::vector<scocg::TuneEntry> tune;   // autotuner decisions of this handle
    // the single-right-hand-side solve that stopped at max_iter and can be
    // continued (scocg_solve_resume): its inputs and the workspace bytes
    // [0, state_bytes) that hold its state
    struct {
        bool ok = false;
        int prec = 0, K = 0, M = 0;
        bool dense = false;
        std::vector<scocg_c128> z;
        std::vector<int64_t> cidx;
        size_t state_bytes = 0;
    } rs;

    void free_all();
    scocg::Layout layout(bool prefer_csr) const;
    double bytes_per_iter(int prec, bool dense_proj, int M) const;
};

namespace scocg {
int cuda_status(cudaError_t e);
// multi-right-hand-side (block) solves (block.cu)
int block_default_tile(int nrhs);
int block_solve(scocg_ctx* h, const scocg_c128* shifts, int K, const void* rhs, int nrhs, const int64_t* proj_idx,
                int M, double tol, scocg_c128* G_out, scocg_info* info, int prec, int T, int per_sm);
int block_autotune(scocg_ctx* h, const scocg_c128* shifts, int K, const void* rhs, int nrhs,
                   const int64_t* proj_idx, int M, double tol, scocg_c128* G_out, int prec, int* T_out,
                   int* per_sm_out);
unsigned long long next_generation();
int init_ctx(scocg_ctx* h, const scocg_opts* opts, void* stream);
void fill_opts(scocg_opts& o, const scocg_opts* in);
int default_seed(const scocg_c128* z, int K);

// Hubbard (hubbard.cu)
cudaError_t hubbard_apply(const Hubbard& hb, int prec, double2 z, const void* x, void* y, cudaStream_t st);
int hubbard_max_ctas(const Hubbard& hb, int prec, int num_sms, size_t dyn_smem = 0);
// real FP64 y = (H - sigma) x - beta x_prev with per-block partials of x^T y (ground state)
cudaError_t hubbard_hx(const Hubbard& hb, const double* x, double* y, const double* xprev, const double* beta,
                       double sigma, const int* skip, double* part, int grid, cudaStream_t st);
template <typename R>
cudaError_t hubbard_launch_solve(const SolveArgs<R>& a, const Hubbard& hb, int grid, cudaStream_t st);
// the two-orbital model (hubbard2.cu), dispatched to from the functions above
cudaError_t hubbard2_apply(const Hubbard& hb, int prec, double2 z, const void* x, void* y, cudaStream_t st);
int hubbard2_max_ctas(const Hubbard& hb, int prec, int num_sms, size_t dyn_smem);
cudaError_t hubbard2_hx(const Hubbard& hb, const double* x, double* y, const double* xprev, const double* beta,
                        double sigma, const int* skip, double* part, int grid, cudaStream_t st);
template <typename R>
cudaError_t hubbard2_launch_solve(const SolveArgs<R>& a, const Hubbard& hb, int grid, cudaStream_t st);

constexpr int kMaxFullShifts = 512;   // shifts per full-vector launch (dynamic shared memory)
int solve_impl(scocg_ctx* h, const scocg_c128* shifts, int nshift, const void* rhs, int nrhs,
               const int64_t* proj_idx, const void* proj_vec, int nproj, double tol, scocg_c128* G_out,
               scocg_info* info, int prec, double2* Xf, double2* Pf, bool resume = false);

// multi-system plans (multi.cu)
void multi_forget(scocg_ctx* h);

// full-vector solve and gradient (adjoint.cu)
int solve_full_impl(scocg_ctx* h, const scocg_c128* shifts, int nshift, const void* rhs, double tol, void* X_out,
                    scocg_info* info);
int grad_impl(scocg_ctx* h, const scocg_c128* shifts, int nshift, const void* rhs, int nrhs,
              const int64_t* proj_idx, const void* proj_vec, int nproj, double tol, const scocg_c128* dL_dG,
              double* dL_dval, scocg_info* info);
}  // namespace scocg
