/*
 * scocg.h -- C ABI of the GB300 shifted-COCG Green's-function library.
 *
 * The library solves, for one real symmetric N x N Hamiltonian H, many complex
 * energies z_k = e_k + i delta_k at once and one or more right-hand sides b,
 *
 *     (z_k I - H) x_k = b                         (arXiv:0802.0748, Eq. lin_eq,
 *                                                  Eq. shift_lin_eq)
 *
 * with the shifted conjugate-orthogonal conjugate-gradient method (Sec. III.C):
 * one seed COCG recurrence on z_s, every other shift obtained from it by scalar
 * recurrences (collinear residuals), seed switching when the seed converges
 * first, and residual monitoring (Eq. residual).  It returns projections
 *
 *     G_mk = c_m^T x_k                            (Eq. gf: G_ij = <i|x_j>)
 *
 * for unit vectors c_m = e_i (Green's-function elements, local DOS
 * -Im G_ii / pi) or dense vectors c_m (for a spectrum <b|G|b> pass c = conj(b)).
 * H is either a CSR matrix (tight-binding form, Sec. II) or the matrix-free
 * extended Hubbard model in a fixed (N_up, N_dn) sector (Sec. IV.B).
 *
 * Conventions for every entry point:
 *  - Complex numbers are (re, im) pairs of doubles, scocg_c128.
 *  - "device" pointers are CUDA global-memory pointers on the handle's device;
 *    "host" pointers are ordinary CPU memory.  Caller memory is only borrowed
 *    for the duration of a call; the library never frees it.
 *  - The handle owns its device copy of H and its workspace (freed by
 *    scocg_destroy).  All device work runs on the stream given at create time
 *    (NULL = legacy default stream); calls that return results synchronise it.
 *  - Errors are reported by return code only (see scocg_status); the library
 *    never exits, aborts or traps.  A handle stays usable after any error
 *    except SCOCG_ERR_CUDA.
 *  - A handle is not thread-safe: one call at a time per handle.
 */
#ifndef SCOCG_H
#define SCOCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct scocg_ctx *scocg_handle;
typedef struct { double re, im; } scocg_c128;

typedef enum {
    SCOCG_OK = 0,               /* all shifts reached the tolerance                 */
    SCOCG_NOT_CONVERGED = 1,    /* max_iter reached; outputs valid, see resid       */
    SCOCG_ERR_INVALID = -1,     /* bad argument (size, pointer, index range)        */
    SCOCG_ERR_CUDA = -2,        /* a CUDA runtime call failed                       */
    SCOCG_ERR_OOM = -3,         /* device allocation failed                         */
    SCOCG_ERR_BREAKDOWN = -4,   /* r^T r, r^T A p or a pi^k became zero / not finite */
    SCOCG_ERR_TIMEOUT = -5,     /* a device-wide barrier did not complete in time   */
    SCOCG_ERR_UNSYMMETRIC = -6, /* CSR input is not structurally/numerically symmetric */
    SCOCG_ERR_TOO_LARGE = -7    /* problem exceeds the fixed scratch of
                                   scocg_solve_csr_noalloc                          */
} scocg_status;

typedef enum {
    SCOCG_FP64 = 0,     /* complex128 vectors, FP64 H values and arithmetic          */
    SCOCG_MIXED = 1,    /* complex64 vectors and FP32 H values with FP32 arithmetic in
                           the H apply and vector updates; FP64 seed scalars, FP64
                           shift recurrences, optional FP64 residual replacement.
                           G carries an error of order eps32 ||H|| / Im z         */
    SCOCG_MIXED_DF = 2  /* compensated FP32: each vector entry is a pair of FP32
                           numbers (hi + lo, about 44 significant bits), FP32 H
                           values, every vector operation in FP32 arithmetic with
                           error-free transformations (TwoSum, FMA TwoProd); FP64
                           seed scalars and shift recurrences.  For Hubbard
                           handles t, U and V enter as float pairs.             */
} scocg_precision;

/* Options, fixed at create time (scocg_set_opts changes them later).
 * A zero-initialised struct (or NULL) selects every default. */
typedef struct {
    int precision;        /* scocg_precision                                          */
    int max_iter;         /* iteration cap per solve; 0 -> 100000                     */
    int replace_every;    /* MIXED: FP64 true-residual replacement of the seed every
                             this many iterations (reliable update of the seed's
                             residual from its compensated solution); 0 or < 0
                             disables it (default).  It does not make complex64
                             vectors accurate: each FP32 apply perturbs the Krylov
                             process itself, which a residual update does not undo
                             (measured: no gain in G).  SCOCG_MIXED_DF is the
                             reduced-precision mode that reaches FP64-like G      */
    int seed;             /* seed shift index; < 0 or out of range -> the seed rule:
                             smallest Im z, then Re z nearest the median Re z, then
                             the lowest index                                         */
    int no_switch;        /* 1 disables seed switching (a converged seed with shifts
                             left then returns SCOCG_ERR_BREAKDOWN)                   */
    int autotune;         /* 1: time the kernel variants on the first solve and keep
                             the fastest for this (N, nnz, nrhs, precision)           */
    double timeout_ms;    /* device barrier watchdog; 0 -> 10000 ms                   */
    int layout;           /* CSR handles: 0 = automatic (4x4-blocked sliced ELL when
                             the pattern allows it, else CSR), 1 = force CSR         */
    int grid;             /* CTAs of the persistent kernel; 0 = automatic, otherwise
                             clamped to the device's co-resident maximum            */
    int debug_inject;     /* fault-injection hook for tests, 0 = off:
                             1 = make one CTA skip one barrier arrival at iteration 3
                                 (the solve must end with SCOCG_ERR_TIMEOUT)
                             2 = poison alpha with NaN at iteration 3 (the solve must
                                 end with SCOCG_ERR_BREAKDOWN)                        */
    int rhs_tile;         /* right-hand sides solved together ("block" mode: one
                             persistent launch in which T slots share every read of
                             H, and a slot whose right-hand side has converged takes
                             the next one).  Used by scocg_solve for CSR handles when
                             nrhs > 1, projections are unit vectors (proj_idx,
                             nproj <= 4) and MIXED residual replacement is off.
                             0 = automatic (the autotuner's choice when autotune = 1,
                             else 8, 16 or 32 by nrhs), 1 = one right-hand side at a
                             time, 8 / 16 / 32 = that many slots                     */
} scocg_opts;

/* Per-solve report.  The two arrays are optional caller-owned HOST buffers of
 * nrhs * nshift entries ([rhs][shift]); set them to NULL to skip. */
typedef struct {
    int iters;             /* seed iterations executed                                */
    int n_switch;          /* seed switches                                          */
    int seed_final;        /* index of the last seed shift                            */
    int n_replace;         /* residual replacements (MIXED)                           */
    long long shift_iters; /* sum over iterations of unconverged (rhs, shift) pairs   */
    int *freeze_iter;      /* out: iteration at which each shift converged (or iters) */
    double *resid;         /* out: ||r_k|| / ||b|| from the recurrence, at the end    */
    double seconds;        /* device time of the solve kernel(s) (CUDA events)        */
    double bytes_per_iter; /* algorithmic bytes of one seed iteration: H once in its
                              device layout plus every vector pass of the kernel     */
} scocg_info;

/*
 * scocg_create_csr -- take a real symmetric H in CSR form (Sec. II tight-binding
 * Hamiltonian; the solver needs (z I - H) complex symmetric, Sec. III.C).
 *   n                 rows (1 <= n < 2^31)
 *   nnz               stored entries
 *   rowptr[n+1]       int64, rowptr[0] = 0, non-decreasing, rowptr[n] = nnz
 *   col[nnz]          int32 column of each entry, 0 <= col < n
 *   val[nnz]          double value of each entry
 *   ptr_on_device     0: the three arrays are host memory; 1: device memory
 *   opts              may be NULL (defaults)
 *   cuda_stream       cudaStream_t for all of this handle's work (NULL = default)
 * The matrix is validated on the device (index range, sorted-or-not is allowed,
 * exact symmetry H_ij == H_ji of every stored entry); a failure returns
 * SCOCG_ERR_INVALID or SCOCG_ERR_UNSYMMETRIC and *out = NULL.  The library
 * copies H into its own device layout (CSR, or 4x4-blocked sliced ELL when the
 * pattern consists of dense 4x4 blocks), with FP32 values in MIXED precision.
 */
int scocg_create_csr(scocg_handle *out, int64_t n, int64_t nnz, const int64_t *rowptr,
                     const int32_t *col, const double *val, int ptr_on_device,
                     const scocg_opts *opts, void *cuda_stream);

/*
 * scocg_create_hubbard -- matrix-free extended Hubbard ring (Sec. IV.B):
 *   H = -t sum_{<ij>,s} (c+_is c_js + h.c.) + U sum_i n_i,up n_i,dn + V sum_<ij> n_i n_j
 * on L sites (2 <= L <= 16) in the sector with n_up up and n_dn down electrons.
 * Bonds are (i, i+1), plus (L-1, 0) when periodic and L >= 3.  Basis index =
 * rank_up * C(L, n_dn) + rank_dn, where rank is the position of the site-
 * occupation bit string (bit i = site i) among all strings with the same number
 * of ones in ascending numeric order.  Fermion signs follow Jordan-Wigner with
 * modes ordered all up-spin sites, then all down-spin sites.
 */
int scocg_create_hubbard(scocg_handle *out, int L, int n_up, int n_dn, double t, double U,
                         double V, int periodic, const scocg_opts *opts, void *cuda_stream);

/*
 * scocg_create_hubbard2 -- matrix-free two-orbital (doubly degenerate)
 * extended Hubbard model on a cluster, the many-electron problem of Sec. IV.B
 * (the paper: N = 8 sites of the sqrt(8) x sqrt(8) square lattice with two
 * orbitals each, N_e = 12, S_z = 0: 64,128,064 states):
 *
 *   H = sum_b sum_{a,a'} sum_s t^b_{aa'} (c+_{i a s} c_{j a' s} + c+_{j a' s} c_{i a s})  (bond b = (i, j))
 *     + U sum_{i,a} n_{ia up} n_{ia dn} + U' sum_i n_{i0} n_{i1} - J sum_{i,s} n_{i0s} n_{i1s}
 *     + J sum_{i,s} c+_{i0s} c+_{i1s'} c_{i0s'} c_{i1s}                          (s' = -s)
 *     + J' sum_i (c+_{i0 up} c+_{i0 dn} c_{i1 dn} c_{i1 up} + h.c.) + V sum_b n_i n_j
 *
 *   n_sites <= 16; n_bonds <= 32, each site in at most 7 bonds;
 *   bond_i, bond_j [n_bonds] host: the sites of each bond (i != j);
 *   bond_t [n_bonds][2][2] host: t^b_{aa'};
 *   n_up, n_dn electrons per spin (each spin sector below 2^23 states).
 * Modes: within a spin 2 i + a (site i, orbital a); all up-spin modes first,
 * then the down-spin ones (Jordan-Wigner order).  Basis index rank_up * D_dn +
 * rank_dn with ranks as in scocg_create_hubbard over the 2 n_sites modes.
 * The handle is a Hubbard handle: scocg_solve, scocg_apply,
 * scocg_ground_state, scocg_krylov_sd accept it, and scocg_excite creates or
 * annihilates mode m = 2 i + a (`site` = m) between two such handles.
 * Returns SCOCG_ERR_INVALID for parameters outside these limits.
 */
int scocg_create_hubbard2(scocg_handle *out, int n_sites, int n_bonds, const int32_t *bond_i,
                          const int32_t *bond_j, const double *bond_t, double U, double Up, double J,
                          double Jp, double V, int n_up, int n_dn, const scocg_opts *opts,
                          void *cuda_stream);

/* Dimension N of the handle's H. */
int scocg_dim(scocg_handle h, int64_t *n);

/* Replace the handle's options (same meaning as at create; precision changes
 * re-layout H on the next solve). */
int scocg_set_opts(scocg_handle h, const scocg_opts *opts);

/*
 * scocg_apply -- y = (z I - H) x once (the matrix of Eq. lin_eq).
 *   precision SCOCG_FP64: x, y device complex128 [N]
 *   precision SCOCG_MIXED: x, y device complex64 [N] (float re, im pairs),
 *                          arithmetic in FP32 with FP32 values of H
 *   precision SCOCG_MIXED_DF: x, y device float4 [N] {re.hi, im.hi, re.lo, im.lo}
 *                          (value = hi + lo), compensated FP32 arithmetic
 * Synchronises the stream.
 */
int scocg_apply(scocg_handle h, scocg_c128 z, const void *x, void *y, int precision);

/*
 * scocg_solve -- shifted COCG for all shifts and right-hand sides (Sec. III.C).
 *   shifts[nshift]        host, z_k (Im z_k > 0 for retarded Green's functions)
 *   rhs                   device complex128 [nrhs][N], b for each right-hand side
 *   proj_idx              host int64 [nrhs][nproj]: c_m = e_{proj_idx} (per rhs), or NULL
 *   proj_vec              device complex128 [nproj][N]: dense c_m shared by all rhs, or NULL
 *                         (exactly one of proj_idx / proj_vec is non-NULL)
 *   tol                   shift k stops once ||r_k|| / ||b|| <= tol, where r_k is the
 *                         residual of Eq. residual tracked by the recurrence
 *   G_out                 device complex128 [nrhs][nproj][nshift], G_mk = c_m^T x_k
 *   info                  optional report (may be NULL)
 * Returns SCOCG_OK, SCOCG_NOT_CONVERGED (outputs valid, per-shift residuals in
 * info) or an error.  1 <= nshift <= 4096, 1 <= nproj <= 32 (<= 4 when nrhs > 1).
 * In block mode (see scocg_opts.rhs_tile) info->iters counts block iterations
 * (each advances every occupied slot by one seed iteration), info->seed_final
 * is the last right-hand side's final seed and info->bytes_per_iter is per
 * block iteration; a right-hand side that breaks down does not stop the others.
 */
int scocg_solve(scocg_handle h, const scocg_c128 *shifts, int nshift, const void *rhs, int nrhs,
                const int64_t *proj_idx, const void *proj_vec, int nproj, double tol,
                scocg_c128 *G_out, scocg_info *info);

/*
 * scocg_solve_resume -- continue the handle's last scocg_solve from where it
 * stopped at max_iter (status SCOCG_NOT_CONVERGED), reusing what was already
 * computed as the seed switch of Sec. III.C does when it carries on with a
 * new seed: the seed vectors r_n and q_n, every shift's recurrence values
 * (pi^k, projected p^k and x^k, freeze state) and the FP64 seed scalars stay
 * in the handle's device workspace, and the continued solve starts from them
 * instead of r_0 = b.
 * The seed iteration count carries on (scocg_set_opts with a larger max_iter
 * caps the total); shifts frozen at the earlier tol stay frozen, the others
 * run to this call's tol.  With the same grid the continued solve equals an
 * uninterrupted one bit for bit.
 *   arguments as scocg_solve with nrhs = 1; shifts (bit for bit), the
 *   projection kind, the unit indices, nproj and the handle's precision must
 *   be those of the stopped solve, and rhs / proj_vec the same data (the
 *   dense projections are read again every iteration)
 * Only one right-hand side solved by the persistent kernel can be continued
 * (not block mode, not scocg_solve_full); any other solve on the handle
 * discards the state.  Returns SCOCG_ERR_INVALID when there is no state to
 * continue or the inputs differ; otherwise as scocg_solve (a continuation
 * that stops at max_iter again can itself be continued).  info->shift_iters
 * and info->seconds count this call's work, info->iters the total.
 */
int scocg_solve_resume(scocg_handle h, const scocg_c128 *shifts, int nshift, const void *rhs,
                       const int64_t *proj_idx, const void *proj_vec, int nproj, double tol,
                       scocg_c128 *G_out, scocg_info *info);

/*
 * Checkpoint of the continuation state on the host (so that a solve can be
 * continued by another process or after the handle was destroyed):
 *   scocg_state_size  bytes of the state of the handle's last stopped solve
 *                     (SCOCG_ERR_INVALID, *bytes = 0, when there is none)
 *   scocg_state_save  copies it into the caller's host buffer (>= that size)
 *   scocg_state_load  makes the buffer the handle's continuation state; the
 *                     next scocg_solve_resume continues from it.  The handle
 *                     must hold the same H (N, nnz and the handle kind are
 *                     checked, the values are not) and have the saved
 *                     precision; SCOCG_ERR_INVALID otherwise.
 * The buffer holds a header, the shifts, the unit projection indices and the
 * device bytes of r_n, q_n (and for SCOCG_MIXED the seed direction and the
 * compensated solution), the per-shift recurrence arrays and the seed
 * scalars.  It is tied to this library's build (no format guarantee).
 */
int scocg_state_size(scocg_handle h, size_t *bytes);
int scocg_state_save(scocg_handle h, void *buf, size_t bytes);
int scocg_state_load(scocg_handle h, const void *buf, size_t bytes);

/*
 * scocg_solve_full -- the same solve for one right-hand side, but every shift's
 * full solution x_k is formed (per-shift vectors p_k, x_k updated each
 * iteration).  X_out: device complex128 [nshift][N].  Used by the adjoint and
 * for true-residual checks; FP64 arithmetic regardless of the precision option.
 */
int scocg_solve_full(scocg_handle h, const scocg_c128 *shifts, int nshift, const void *rhs,
                     double tol, void *X_out, scocg_info *info);

/*
 * scocg_grad -- gradient of a real loss L(G) with respect to every stored CSR
 * value, given dL_dG (device complex128 [nrhs][nproj][nshift], torch
 * convention dL/dRe G + i dL/dIm G).  With A_k = z_k I - H, x_k = A_k^{-1} b
 * and y_mk = A_k^{-1} c_m (A_k is complex symmetric, so the adjoint solve is a
 * second forward solve with the projection vectors as right-hand sides):
 *   dL_dval[v] = Re sum_{k,m} conj(dL_dG_mk) y_mk[a] x_k[b]   for entry v = (a, b)
 * Each stored entry is treated as an independent parameter; the gradient of a
 * symmetric pair (a,b),(b,a) is dL_dval[(a,b)] + dL_dval[(b,a)].
 * dL_dval: device double [nnz], overwritten.  Shifts are processed in chunks
 * when the [chunk][N] solution vectors do not fit.  Not available for Hubbard
 * handles (SCOCG_ERR_INVALID).  nrhs must be 1.
 */
int scocg_grad(scocg_handle h, const scocg_c128 *shifts, int nshift, const void *rhs, int nrhs,
               const int64_t *proj_idx, const void *proj_vec, int nproj, double tol,
               const scocg_c128 *dL_dG, double *dL_dval, scocg_info *info);

/*
 * scocg_density -- density-matrix elements by the Fermi integral of Eq. densityM:
 *   rho_m = -(1/pi) int de Im G_m(e + i delta) f((e - mu) / kT)
 * taken on the uniform real-axis grid e_k = emin + k (emax - emin) / (nquad - 1),
 * k < nquad, with trapezoid weights, where G_m(z) = c_m^T (z I - H)^{-1} b comes
 * from one shifted-COCG solve on the shifts e_k + i delta (the block or the
 * one-right-hand-side path of scocg_solve, same rhs / projection conventions).
 * This is the projected density matrix c_m^T rho b when the eigenstate weights
 * (c_m^T phi)(phi^T b) are real (unit vectors, or c = conj(b)); delta > 0
 * broadens it by a Lorentzian (error O(delta / kT)), and the window should
 * cover the spectrum with a margin of several delta.
 *   mu, kT       chemical potential and k_B T (kT >= 0; kT = 0 is the step)
 *   delta        broadening, > 0
 *   emin < emax  energy window;  2 <= nquad <= 4096
 *   rho_out      device double [nrhs][nproj], written
 * Returns what the solve returns (SCOCG_NOT_CONVERGED leaves rho valid).
 * Allocates a device buffer for the intermediate G.
 */
int scocg_density(scocg_handle h, double mu, double kT, double delta, double emin, double emax, int nquad,
                  const void *rhs, int nrhs, const int64_t *proj_idx, const void *proj_vec, int nproj,
                  double tol, double *rho_out, scocg_info *info);

/*
 * scocg_solve_multi -- several independent solves (systems of different sizes,
 * one right-hand side each) in ONE cooperative launch: the GPU's co-resident
 * CTAs are split among the systems (at least enough for each system's shifts,
 * otherwise in proportion to its rows) and each system keeps its own barrier
 * counter, partial sums and seed scalars.  Per system s:
 *   hs[s]                CSR handle (all: same device, stream, precision and
 *                        device layout kind)
 *   shifts[s][nshift[s]] host shifts; rhs[s] device complex128 [N_s]
 *   proj_idx[s][nproj[s]] host unit projections, or proj_vec[s] device
 *                        complex128 [nproj[s]][N_s] (one of the two arrays of
 *                        pointers is NULL)
 *   G_out[s]             device complex128 [nproj[s]][nshift[s]]
 *   info                 optional, [nsys] reports (seconds = the whole launch)
 * use_graph = 1 captures the control-block resets and the launch into a CUDA
 * graph on the first call and replays it while the handles, sizes and buffer
 * pointers stay the same (shift values may change; they are copied before
 * each replay).  One plan is cached per process; scocg_multi_release frees it.
 * Returns the worst status over the systems.
 */
int scocg_solve_multi(int nsys, const scocg_handle *hs, const scocg_c128 *const *shifts, const int *nshift,
                      const void *const *rhs, const int64_t *const *proj_idx, const void *const *proj_vec,
                      const int *nproj, double tol, scocg_c128 *const *G_out, scocg_info *info, int use_graph);

/* Free the cached multi-system plan (and its CUDA graph), if any. */
void scocg_multi_release(void);

/*
 * scocg_solve_csr_noalloc -- the FP64 solve of scocg_solve for one right-hand
 * side, for callers that cannot allocate device memory when they solve (an
 * application whose memory pool or arena owns all device memory, a real-time
 * loop that must not take the allocator's locks, a host that reserves all
 * memory up front).  It takes no handle and allocates nothing: no cudaMalloc,
 * no cudaFree, no allocating library call.  The paper has no counterpart; this
 * is an interface for such callers.
 *
 * Inputs and outputs belong to the caller:
 *   n, nnz, rowptr[n+1] (device int32), col[nnz] (device int32), val[nnz]
 *                        (device double): H in CSR; NOT validated -- H must be
 *                        real symmetric with in-range indices (a bounds-checked
 *                        build, -DSCOCG_CHECKED, skips an out-of-range index
 *                        and returns SCOCG_ERR_INVALID)
 *   shifts[nshift]       host; rhs device complex128 [n]
 *   proj_idx[nproj] host int64 | proj_vec device complex128 [nproj][n]
 *   tol, max_iter (0 -> 100000), G_out device complex128 [nproj][nshift],
 *   info (optional; info->seconds is 0), cuda_stream (NULL = default stream).
 * The solve's scratch (r, q, per-shift state, partial sums, control block)
 * lives in one fixed device array of 24 MiB compiled into the library, which
 * every GPU that loads the library holds until the process exits.  Problems
 * whose scratch does not fit return SCOCG_ERR_TOO_LARGE: about
 * 2 * 16 * n + 120 * nshift * (1 + nproj) bytes plus ~40 KB, i.e. n up to
 * about 780,000 rows at a few hundred shifts.
 * The first call on a device looks the array's device address up with
 * cudaGetSymbolAddress (with that device current) and keeps it together with
 * the id of the current CUDA context; a call in another context (after
 * cudaDeviceReset, for instance) looks it up again.  Make the first call in
 * each context before any stream capture.  Every call reuses the same array and leaves its
 * contents behind (the call clears what must start at zero), so calls whose
 * work overlaps on the GPU -- from several threads or streams -- race: issue
 * them one after another.
 */
int scocg_solve_csr_noalloc(int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                            const double *val, const scocg_c128 *shifts, int nshift, const void *rhs,
                            const int64_t *proj_idx, const void *proj_vec, int nproj, double tol,
                            int max_iter, scocg_c128 *G_out, scocg_info *info, void *cuda_stream);

/*
 * scocg_ground_state -- lowest eigenvalue E and unit eigenvector psi of the
 * real symmetric H of a CSR or Hubbard handle, by the cycle of Sec. II.B: the
 * Lanczos method (its basis loses orthogonality; it is not reorthogonalized),
 * then the conjugate-gradient method used as inverse iteration, repeated until
 * the residual norm is small enough.  One cycle:
 *   m Lanczos steps from psi (fewer when beta_j vanishes), kept in device
 *   memory as V[m][N]; (theta, s) = lowest eigenpair of the tridiagonal T;
 *   psi = V s / ||V s||; E = psi^T H psi; res = ||H psi - E psi||_2;
 *   done when res <= tol; else (not in the last cycle) CG on
 *   (H - sigma) y = psi, sigma = E - res, from y = 0 for at most cg_steps
 *   steps (ended earlier at a relative residual of 1e-10 or when
 *   p^T (H - sigma) p <= 0), and psi = y / ||y|| (kept if y = 0).
 * FP64 arithmetic regardless of the handle's precision option.
 *   v0           device double [N], start vector (not zero; caller-owned)
 *   psi          device double [N], written: the eigenvector (sign arbitrary)
 *   m            Lanczos steps per cycle, 2..1024 (clamped to N); the basis
 *                needs (m + 5) N doubles of device memory, allocated per call
 *   cg_steps     CG steps per inverse iteration, >= 0 (0: restart from the
 *                Ritz vector alone)
 *   max_cycles   >= 1
 *   tol          residual bound, >= 0
 *   energy       host double, written: E = psi^T H psi of the returned psi
 *   info         optional, written
 * Returns SCOCG_OK, SCOCG_NOT_CONVERGED (psi, E and info->residual are those
 * of the last cycle), SCOCG_ERR_BREAKDOWN (a non-finite E or residual),
 * SCOCG_ERR_INVALID, SCOCG_ERR_OOM or SCOCG_ERR_CUDA.
 */
typedef struct {
    int cycles;               /* Lanczos / inverse-iteration cycles run               */
    long long lanczos_steps;  /* Lanczos steps over all cycles (one H apply each)     */
    long long cg_steps;       /* CG steps over all inverse iterations (one apply each) */
    double residual;          /* ||H psi - E psi||_2 of the returned psi              */
    double seconds;           /* device time from the first to the last kernel        */
    double bytes_per_step;    /* algorithmic bytes of one Lanczos step: H once in its
                                 device layout plus 8 FP64 vector passes              */
} scocg_ground_info;

int scocg_ground_state(scocg_handle h, const double *v0, double *psi, int m, int cg_steps, int max_cycles,
                       double tol, double *energy, scocg_ground_info *info);

/*
 * scocg_excite -- one-particle excitation vector between Hubbard sectors
 * (Sec. IV.B: the ionization and affinity spectra are G(z) = b^T (z - H)^{-1} b
 * for b = c_{i s}|psi_0> and b = c+_{i s}|psi_0>):
 *   out = c_{site,spin} psi   (create = 0; to = sector with one spin-s electron less)
 *   out = c+_{site,spin} psi  (create = 1; to = sector with one spin-s electron more)
 * with modes ordered all up sites then all down sites (the Jordan-Wigner
 * convention of the Hubbard handles' hopping signs).  from / to: Hubbard
 * handles with the same L whose sectors differ by exactly that electron
 * (else SCOCG_ERR_INVALID); spin 0 = up, 1 = down; 0 <= site < L.
 *   psi   device double [N_from]
 *   out   device complex128 [N_to], written (imaginary parts 0), ready as the
 *         right-hand side of scocg_solve (spectrum: proj_vec = out, since
 *         conj(b) = b)
 * Runs on to's stream (after from's stream has finished, if they differ) and
 * synchronises it.
 */
int scocg_excite(scocg_handle from, scocg_handle to, int site, int spin, int create, const double *psi,
                 void *out);

/*
 * scocg_krylov_sd -- Green's functions by subspace diagonalisation in the
 * Krylov subspace K_nu(H, b) (Sec. III.B, Eq. Ham_in_KS), the cheaper
 * estimator that the shifted COCG method refines: nu Lanczos steps from b (no
 * reorthogonalization; fewer steps when beta_j vanishes) give the reduced
 * Hamiltonian T (tridiagonal) and the projections c_m^T v_j; T's eigenpairs
 * (e_a, s_a) give the approximate eigenvectors w_a = sum_j s_a(j) v_j and
 *   G_m(z_k) = sum_a weight[m][a] / (z_k - e_a),
 *   weight[m][a] = (c_m^T w_a)(w_a^T b) = (sum_j s_a(j) c_m^T v_j) ||b|| s_a(0).
 * FP64 arithmetic regardless of the handle's precision option; CSR or Hubbard
 * handle.  On the 4x4-blocked layout with unit projections the recursion runs
 * as one cooperative launch (two CTAs per SM, or the handle's grid option if
 * smaller; its grid barriers give up after the handle's timeout_ms with
 * SCOCG_ERR_TIMEOUT).  The eigenvalues come from bisection on the Sturm count, the
 * eigenvectors from inverse iteration, orthogonalised within clusters of
 * eigenvalues closer than 1e-3 ||T|| (where the lost orthogonality puts the
 * ghost copies of converged eigenvalues).  A density-matrix element follows
 * as sum_a f(e_a) weight[m][a].
 *   b            device double [N] (real, not zero)
 *   nu           1..1024 Lanczos steps
 *   shifts       host [nshift] (1..2^20)
 *   proj_idx     host int64 [nproj] unit projections e_i, OR
 *   proj_vec     device double [nproj][N] real projection vectors; 1 <= nproj <= 64
 *   G_out        device complex128 [nproj][nshift], written
 *   ritz         device double [nu] or NULL: the eigenvalues e_a, ascending
 *                (the first *nu_used are written)
 *   weight       device double [nproj][nu] or NULL (row stride nu; the first
 *                *nu_used of each row are written)
 *   nu_used      host int or NULL: Lanczos steps done
 *   seconds      host double or NULL: device time
 * Allocates about (4 N + 6 nu^2 + 2 nproj nu) doubles of device memory per call.
 * Returns SCOCG_OK, SCOCG_ERR_INVALID (also for b = 0), SCOCG_ERR_OOM or
 * SCOCG_ERR_CUDA.
 */
int scocg_krylov_sd(scocg_handle h, const double *b, int nu, const scocg_c128 *shifts, int nshift,
                    const int64_t *proj_idx, const double *proj_vec, int nproj, scocg_c128 *G_out,
                    double *ritz, double *weight, int *nu_used, double *seconds);

/*
 * scocg_krylov_sd_multi -- scocg_krylov_sd for several right-hand sides with
 * unit projections (e.g. the local Green's functions G_jj of many sites):
 * B[r] is right-hand side r, its projections e_{proj_idx[r][m]}.  On the
 * 4x4-blocked layout (CSR handles whose pattern allows it) up to 32 of them
 * run as one cooperative launch whose Lanczos vectors are [N][T] (T = 8, 16
 * or 32 slots, the right-hand side fastest), so that every read of H serves
 * T recursions, each with its own scalars and end; other handles run the
 * single-right-hand-side recursion once per right-hand side.  Each slot does
 * the same arithmetic as scocg_krylov_sd (its partial sums run in another
 * order), in FP64, or for a handle with precision SCOCG_MIXED_DF in
 * compensated FP32 (H's FP32 blocks, vector entries as float pairs hi + lo
 * with error-free products and sums, FP64 step scalars), which runs on the
 * FP32 pipe instead of the FP64 one.
 *   B            device double [nrhs][N] (each real and not zero)
 *   proj_idx     host int64 [nrhs][nproj], 1 <= nproj <= 64
 *   G_out        device complex128 [nrhs][nproj][nshift], written
 *   nu_used      host int [nrhs] or NULL: Lanczos steps done per right-hand side
 *   seconds      host double or NULL: device time
 * nu and shifts as in scocg_krylov_sd.  Allocates about (5 T N + T (2 + nproj)
 * nu + 6 nu^2) doubles of device memory per call.  Returns SCOCG_OK,
 * SCOCG_ERR_INVALID (also when a right-hand side is zero), SCOCG_ERR_TIMEOUT,
 * SCOCG_ERR_OOM or SCOCG_ERR_CUDA.
 */
int scocg_krylov_sd_multi(scocg_handle h, const double *B, int nrhs, int nu, const scocg_c128 *shifts,
                          int nshift, const int64_t *proj_idx, int nproj, scocg_c128 *G_out, int *nu_used,
                          double *seconds);

/* Free the handle and everything it owns (NULL is ignored). */
void scocg_destroy(scocg_handle h);

/* Static description of a status code. */
const char *scocg_strerror(int code);

/*
 * scocg_hubbard_tables -- copy the per-spin basis tables built on the device by
 * scocg_create_hubbard, for checking.  Arrays are host memory:
 *   states[D]            bit string of each rank (D = C(L, n_s))
 *   hop_target[D][2L]    rank reached by each hop (-1 = unused slot)
 *   hop_sign[D][2L]      Jordan-Wigner sign (+1/-1) of that hop (0 = unused)
 * spin 0 = up, 1 = down.  Returns D in *dim.
 */
int scocg_hubbard_tables(scocg_handle h, int spin, int32_t *dim, uint32_t *states,
                         int32_t *hop_target, int8_t *hop_sign);

#ifdef __cplusplus
}
#endif
#endif /* SCOCG_H */
