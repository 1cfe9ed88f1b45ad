/*
 * CPU oracle for the shifted-COCG Green's-function solver.  TEST
 * INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
 * the benchmark call it; the product path never does.  It shares no code with
 * the CUDA path.
 *
 * Everything here is plain double-precision C, written for reading, not speed:
 * full per-shift solution and direction vectors, one step at a time, in the
 * order the method states them.  OpenMP only splits independent loops (rows
 * of a matrix-vector product, shifts of the per-shift update); every sum runs
 * in a fixed sequential order, so results do not depend on the thread count.
 *
 * Paper: Fujiwara, Hoshi, Yamamoto, "Theory of large-scale matrix computation
 * and applications to electronic structure calculation" (arXiv:0802.0748).
 *   Eq. (gf)          G_ij(e) = [(e + i delta - H)^{-1}]_ij
 *   Eq. (lin_eq)      [(e + i delta) 1 - H] |x_j> = |j>
 *   Eq. (inv_KS)      K_nu(H, |j>) = K_nu(sigma 1 + H, |j>)
 *   Sec. III.C        COCG for the complex-symmetric (e0 + i delta) 1 - H,
 *                     shifted systems (Eq. shift_lin_eq) through collinear
 *                     residuals, seed switching
 *   Eq. (residual)    |r> = (e + i delta - H)|x> - |j>, monitored to stop
 *   Sec. IV.B         extended Hubbard model in a fixed-S_z sector
 *
 * The paper states what shifted COCG does but prints no recurrence.  The
 * recurrences below are those of textbook COCG (van der Vorst & Melissen 1990)
 * combined with the collinear-residual property the paper states: residual
 * polynomials R_n with R_n(0) = 1 satisfy a three-term recurrence, and the
 * residual of the shifted system z_k is r_n / pi^k_n with pi^k_n = R_n(-sigma_k).
 *
 * Functions whose result has no closed-form pin of its own are pinned by the
 * tests through dense LU, closed forms, invariants and exact diagonalisation.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum {
    OR_OK = 0, OR_NOT_CONVERGED = 1, OR_ERR_INVALID = -1, OR_ERR_OOM = -3, OR_ERR_BREAKDOWN = -4,
};

/* ------------------------------------------------------------------------ */
/* y = (z I - H) x for a real CSR matrix H and complex x (Eq. lin_eq's matrix). */
static void apply_shifted(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                          cplx z, const cplx *x, cplx *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        cplx hx = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
            hx += val[e] * x[col[e]];
        y[i] = z * x[i] - hx;
    }
}

/* Bilinear form u^T v (no conjugation): the inner product COCG uses for a
 * complex-symmetric matrix (Sec. III.C). */
static cplx dot_t(int64_t n, const cplx *u, const cplx *v)
{
    cplx s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += u[i] * v[i];
    return s;
}

/* Euclidean 2-norm with conjugation, used for residual monitoring (Eq. residual). */
static double norm2(int64_t n, const cplx *u)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += creal(u[i]) * creal(u[i]) + cimag(u[i]) * cimag(u[i]);
    return sqrt(s);
}

/* The seed rule (the paper leaves the choice open): smallest Im z; ties go to
 * Re z closest to the median of all Re z; remaining ties to the lowest index. */
static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

int oracle_default_seed(int nshift, const double *z)
{
    if (nshift <= 0) return -1;
    double *re = malloc(sizeof(double) * nshift);
    if (!re) return -1;
    for (int k = 0; k < nshift; ++k) re[k] = z[2 * k];
    qsort(re, nshift, sizeof(double), cmp_double);
    double med = (nshift % 2) ? re[nshift / 2] : 0.5 * (re[nshift / 2 - 1] + re[nshift / 2]);
    free(re);
    int best = 0;
    for (int k = 1; k < nshift; ++k) {
        double ik = z[2 * k + 1], ib = z[2 * best + 1];
        if (ik < ib) { best = k; continue; }
        if (ik == ib && fabs(z[2 * k] - med) < fabs(z[2 * best] - med)) best = k;
    }
    return best;
}

/*
 * Shifted COCG for one right-hand side b and all shifts z_k at once
 * (Sec. III.C, Eqs. lin_eq and shift_lin_eq), keeping full per-shift vectors.
 *
 * Seed s, A = z_s I - H.  x = 0, r_0 = b, rho_0 = r_0^T r_0, beta_{-1} = 0,
 * alpha_{-1} = 1, pi^k_{-1} = pi^k_0 = 1, sigma_k = z_k - z_s.  Iteration n:
 *   beta^k_{n-1} = (pi^k_{n-1} / pi^k_n)^2 beta_{n-1}
 *   p^k_n        = r_n / pi^k_n + beta^k_{n-1} p^k_{n-1}      (seed: pi = 1)
 *   q_n          = A p^s_n,   alpha_n = rho_n / (p^s_n^T q_n)
 *   pi^k_{n+1}   = (1 + alpha_n sigma_k) pi^k_n
 *                  + (alpha_n beta_{n-1} / alpha_{n-1}) (pi^k_n - pi^k_{n-1})
 *   alpha^k_n    = (pi^k_n / pi^k_{n+1}) alpha_n
 *   x^k_{n+1}    = x^k_n + alpha^k_n p^k_n
 *   r_{n+1}      = r_n - alpha_n q_n,  rho_{n+1} = r_{n+1}^T r_{n+1},
 *   beta_n       = rho_{n+1} / rho_n
 * Residual of shift k (collinear residuals): r_{n+1} / pi^k_{n+1}; shift k is
 * frozen (no further update, output kept) once
 * ||r_{n+1}|| / (|pi^k_{n+1}| ||b||) <= tol (Eq. residual monitoring).
 *
 * Seed switching (Sec. III.C): when the seed shift has converged and others
 * have not, the unconverged shift with the largest residual becomes the seed
 * s' and the run continues with the same Krylov information:
 *   r <- r_{n+1} / pi^{s'}_{n+1},  rho <- rho_{n+1} / (pi^{s'}_{n+1})^2,
 *   alpha_n <- alpha^{s'}_n,  beta_n <- beta^{s'}_n,
 *   pi^k_j <- pi^k_j / pi^{s'}_j (j = n, n+1),  sigma_k <- z_k - z_{s'};
 * the per-shift vectors x^k, p^k are unchanged.
 *
 * Arguments (all host memory, complex numbers as (re, im) double pairs):
 *   n, rowptr[n+1], col[nnz], val[nnz]   real symmetric H in CSR
 *   nshift, z[nshift]                    shifts z_k
 *   b[n]                                 right-hand side
 *   nproj, proj_idx[nproj] | proj_vec[nproj][n]   projections c_m (e_i or dense)
 *   tol, max_iter                        stopping rule (tol <= 0: never freeze)
 *   seed                                 seed shift index, or -1 for the rule above
 *   allow_switch                         0 disables seed switching
 *   G[nproj][nshift]                     out: G_mk = c_m^T x^k
 *   iters[nshift]                        out: iteration count at freeze (or total)
 *   resid[nshift]                        out: ||r^k|| / ||b|| at the end
 *   X[nshift][n] (may be NULL)           out: full solutions x^k
 *   r_out[n], pi_out[nshift] (may be NULL) out: final seed residual and pi^k
 *   stats[4] (may be NULL)               out: total iterations, shift-iterations,
 *                                        number of switches, final seed index
 * Returns OR_OK, OR_NOT_CONVERGED (max_iter reached), or an error code.
 */
int oracle_shifted_cocg(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                        int nshift, const double *z_in, const double *b_in,
                        int nproj, const int64_t *proj_idx, const double *proj_vec_in,
                        double tol, int max_iter, int seed, int allow_switch,
                        double *G_out, int *iters, double *resid, double *X_out,
                        double *r_out, double *pi_out, double *stats)
{
    if (n <= 0 || nshift <= 0 || max_iter < 0) return OR_ERR_INVALID;
    const cplx *z = (const cplx *)z_in;
    const cplx *b = (const cplx *)b_in;
    const cplx *proj_vec = (const cplx *)proj_vec_in;
    if (seed < 0) seed = oracle_default_seed(nshift, z_in);
    if (seed < 0 || seed >= nshift) return OR_ERR_INVALID;

    cplx *r = malloc(sizeof(cplx) * n);
    cplx *q = malloc(sizeof(cplx) * n);
    cplx *x = calloc((size_t)nshift * n, sizeof(cplx));
    cplx *p = calloc((size_t)nshift * n, sizeof(cplx));
    cplx *pi_prev = malloc(sizeof(cplx) * nshift);
    cplx *pi_cur = malloc(sizeof(cplx) * nshift);
    cplx *pi_next = malloc(sizeof(cplx) * nshift);
    cplx *sigma = malloc(sizeof(cplx) * nshift);
    cplx *alpha_k = malloc(sizeof(cplx) * nshift);
    char *frozen = calloc(nshift, 1);
    if (!r || !q || !x || !p || !pi_prev || !pi_cur || !pi_next || !sigma || !alpha_k || !frozen) {
        free(r); free(q); free(x); free(p); free(pi_prev); free(pi_cur); free(pi_next);
        free(sigma); free(alpha_k); free(frozen);
        return OR_ERR_OOM;
    }

    memcpy(r, b, sizeof(cplx) * n);
    const double bnorm = norm2(n, b);
    for (int k = 0; k < nshift; ++k) {
        pi_prev[k] = 1.0; pi_cur[k] = 1.0; sigma[k] = z[k] - z[seed];
        iters[k] = 0; resid[k] = 1.0;
    }
    cplx rho = dot_t(n, r, r);
    cplx alpha_prev = 1.0, beta_prev = 0.0;
    long long shift_iters = 0;
    int n_switch = 0, status = OR_NOT_CONVERGED, it = 0;

    if (bnorm == 0.0) {                     /* b = 0: x = 0 solves every shift */
        for (int k = 0; k < nshift; ++k) { frozen[k] = 1; resid[k] = 0.0; }
        status = OR_OK;
    }

    for (it = 0; status == OR_NOT_CONVERGED && it < max_iter; ++it) {
        cplx *ps = p + (size_t)seed * n;
        int nactive = 0;
        for (int k = 0; k < nshift; ++k) nactive += !frozen[k];
        shift_iters += nactive;

        /* p^k_n = r_n / pi^k_n + beta^k_{n-1} p^k_{n-1} for every unfrozen shift */
#pragma omp parallel for schedule(dynamic)
        for (int k = 0; k < nshift; ++k) {
            if (frozen[k]) continue;
            cplx ratio = pi_prev[k] / pi_cur[k];
            cplx beta_k = ratio * ratio * beta_prev;
            cplx inv_pi = 1.0 / pi_cur[k];
            cplx *pk = p + (size_t)k * n;
            for (int64_t i = 0; i < n; ++i) pk[i] = r[i] * inv_pi + beta_k * pk[i];
        }

        /* q_n = A p_n and alpha_n = rho_n / (p_n^T q_n) for the seed */
        apply_shifted(n, rowptr, col, val, z[seed], ps, q);
        cplx pq = dot_t(n, ps, q);
        if (pq == 0.0 || rho == 0.0) { status = OR_ERR_BREAKDOWN; break; }
        cplx alpha = rho / pq;

        /* pi^k_{n+1}, alpha^k_n, x^k_{n+1} */
        int bad_pi = 0;
        for (int k = 0; k < nshift; ++k) {
            if (frozen[k]) continue;
            pi_next[k] = (1.0 + alpha * sigma[k]) * pi_cur[k]
                       + (alpha * beta_prev / alpha_prev) * (pi_cur[k] - pi_prev[k]);
            if (pi_next[k] == 0.0) bad_pi = 1;
            else alpha_k[k] = pi_cur[k] / pi_next[k] * alpha;
        }
        if (bad_pi) { status = OR_ERR_BREAKDOWN; break; }
#pragma omp parallel for schedule(dynamic)
        for (int k = 0; k < nshift; ++k) {
            if (frozen[k]) continue;
            cplx *xk = x + (size_t)k * n, *pk = p + (size_t)k * n;
            for (int64_t i = 0; i < n; ++i) xk[i] += alpha_k[k] * pk[i];
        }
        for (int k = 0; k < nshift; ++k) {
            if (frozen[k]) continue;
            pi_prev[k] = pi_cur[k]; pi_cur[k] = pi_next[k];
        }

        /* r_{n+1} = r_n - alpha_n q_n, rho_{n+1}, beta_n */
        for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];
        cplx rho_next = dot_t(n, r, r);
        cplx beta = rho_next / rho;
        rho = rho_next; alpha_prev = alpha; beta_prev = beta;

        /* residual monitoring: ||r^k_{n+1}|| / ||b|| = ||r_{n+1}|| / (|pi^k_{n+1}| ||b||) */
        double rnorm = norm2(n, r);
        int remaining = 0;
        for (int k = 0; k < nshift; ++k) {
            if (frozen[k]) continue;
            resid[k] = rnorm / (cabs(pi_cur[k]) * bnorm);
            iters[k] = it + 1;
            if (tol > 0.0 && resid[k] <= tol) frozen[k] = 1;
            else ++remaining;
        }
        if (remaining == 0) { status = OR_OK; ++it; break; }
        if (frozen[seed]) {
            if (!allow_switch) { status = OR_ERR_BREAKDOWN; break; }
            /* seed switching: the unconverged shift with the largest residual */
            int s2 = -1;
            for (int k = 0; k < nshift; ++k)
                if (!frozen[k] && (s2 < 0 || cabs(pi_cur[k]) < cabs(pi_cur[s2]))) s2 = k;
            cplx pn = pi_prev[s2], pn1 = pi_cur[s2];
            for (int64_t i = 0; i < n; ++i) r[i] /= pn1;
            rho = rho / (pn1 * pn1);
            alpha_prev = alpha_k[s2];
            beta_prev = beta * (pn / pn1) * (pn / pn1);
            for (int k = 0; k < nshift; ++k) {
                pi_prev[k] /= pn; pi_cur[k] /= pn1; sigma[k] = z[k] - z[s2];
            }
            pi_prev[s2] = 1.0; pi_cur[s2] = 1.0;   /* exact for the new seed */
            seed = s2;
            ++n_switch;
        }
    }

    /* G_mk = c_m^T x^k (Eq. gf with <i| = c_m^T) */
    for (int m = 0; m < nproj; ++m)
        for (int k = 0; k < nshift; ++k) {
            const cplx *xk = x + (size_t)k * n;
            cplx g;
            if (proj_idx) g = xk[proj_idx[m]];
            else g = dot_t(n, proj_vec + (size_t)m * n, xk);
            ((cplx *)G_out)[(size_t)m * nshift + k] = g;
        }
    if (X_out) memcpy(X_out, x, sizeof(cplx) * (size_t)nshift * n);
    if (r_out) memcpy(r_out, r, sizeof(cplx) * n);
    if (pi_out) memcpy(pi_out, pi_cur, sizeof(cplx) * nshift);
    if (stats) { stats[0] = it; stats[1] = (double)shift_iters; stats[2] = n_switch; stats[3] = seed; }

    free(r); free(q); free(x); free(p); free(pi_prev); free(pi_cur); free(pi_next);
    free(sigma); free(alpha_k); free(frozen);
    return status;
}

/* y = (z I - H) x, exposed for the tests (Eq. lin_eq's matrix applied once). */
void oracle_apply_shifted(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                          double z_re, double z_im, const double *x, double *y)
{
    apply_shifted(n, rowptr, col, val, z_re + I * z_im, (const cplx *)x, (cplx *)y);
}

/* ------------------------------------------------------------------------ */
/* Extended Hubbard model in a fixed (N_up, N_dn) sector (Sec. IV.B).
 *
 *   H = -t sum_{<ij>, s} (c+_{is} c_{js} + c+_{js} c_{is})
 *       + U sum_i n_{i up} n_{i dn} + V sum_{<ij>} n_i n_j,   n_i = n_{i up} + n_{i dn}
 *
 * Bonds: (i, i+1) for i < L-1, plus (L-1, 0) when periodic and L >= 3.
 * Fock modes are ordered all up-spin sites 0..L-1, then all down-spin sites
 * 0..L-1; a basis state is the product of creation operators in that mode order
 * acting on the vacuum.  Each operator's sign is taken literally from the
 * Jordan-Wigner definition: c_m and c+_m pick up (-1)^(number of occupied modes
 * before m).  Basis order: index = rank_up * D_dn + rank_dn, where rank is the
 * position of the bit string among all L-bit strings of the same popcount in
 * ascending numeric order.  Ranks are found by enumerating all 2^L strings.
 * ------------------------------------------------------------------------ */

static int popcount_u32(uint32_t v) { int c = 0; while (v) { c += v & 1u; v >>= 1; } return c; }

/* Fermion sign of c_m on a 2L-mode occupation word (bit m = mode m). */
static int jw_sign_before(uint64_t occ, int m)
{
    int c = 0;
    for (int j = 0; j < m; ++j) c += (int)((occ >> j) & 1u);
    return (c & 1) ? -1 : 1;
}

/* Number of states with popcount k among L-bit strings (the sector size per spin). */
int64_t oracle_sector_dim(int L, int k)
{
    int64_t count = 0;
    for (uint32_t s = 0; s < (1u << L); ++s) count += popcount_u32(s) == k;
    return count;
}

/* Builds H of the sector as CSR.  Call once with rowptr/col/val NULL to get
 * *nnz_out (returned) and once with arrays sized [dim+1], [nnz], [nnz].
 * Entries within a row are sorted by column; exact zeros are not stored. */
int64_t oracle_hubbard_csr(int L, int n_up, int n_dn, double t, double U, double V, int periodic,
                           int64_t *rowptr, int32_t *col, double *val)
{
    if (L < 2 || L > 20 || n_up < 0 || n_dn < 0 || n_up > L || n_dn > L) return -1;
    const uint32_t full = 1u << L;
    int32_t *rank = malloc(sizeof(int32_t) * full);
    uint32_t *up_states = malloc(sizeof(uint32_t) * full);
    uint32_t *dn_states = malloc(sizeof(uint32_t) * full);
    if (!rank || !up_states || !dn_states) { free(rank); free(up_states); free(dn_states); return -3; }
    int64_t Du = 0, Dd = 0;
    for (uint32_t s = 0; s < full; ++s) {
        rank[s] = -1;
        if (popcount_u32(s) == n_up) up_states[Du++] = s;
        if (popcount_u32(s) == n_dn) dn_states[Dd++] = s;
    }
    int32_t *rank_up = malloc(sizeof(int32_t) * full), *rank_dn = malloc(sizeof(int32_t) * full);
    if (!rank_up || !rank_dn) { free(rank); free(up_states); free(dn_states); free(rank_up); free(rank_dn); return -3; }
    for (uint32_t s = 0; s < full; ++s) { rank_up[s] = -1; rank_dn[s] = -1; }
    for (int64_t i = 0; i < Du; ++i) rank_up[up_states[i]] = (int32_t)i;
    for (int64_t i = 0; i < Dd; ++i) rank_dn[dn_states[i]] = (int32_t)i;

    int nb = 0, bi[64], bj[64];
    for (int i = 0; i + 1 < L; ++i) { bi[nb] = i; bj[nb] = i + 1; ++nb; }
    if (periodic && L >= 3) { bi[nb] = L - 1; bj[nb] = 0; ++nb; }

    const int64_t dim = Du * Dd;
    int64_t nnz = 0;
    /* per row: at most 1 diagonal + 2 * nb * 2 hops */
    int64_t cap = 1 + 4 * nb;
    int32_t *rc = malloc(sizeof(int32_t) * cap);
    double *rv = malloc(sizeof(double) * cap);
    if (!rc || !rv) { free(rank); free(up_states); free(dn_states); free(rank_up); free(rank_dn); free(rc); free(rv); return -3; }

    if (rowptr) rowptr[0] = 0;
    for (int64_t iu = 0; iu < Du; ++iu) {
        for (int64_t id = 0; id < Dd; ++id) {
            const uint32_t u = up_states[iu], d = dn_states[id];
            const uint64_t occ = (uint64_t)u | ((uint64_t)d << L);
            int cnt = 0;
            /* diagonal: U n_up n_dn + V n_i n_j */
            double diag = 0.0;
            for (int i = 0; i < L; ++i) diag += U * (double)(((u >> i) & 1u) * ((d >> i) & 1u));
            for (int e = 0; e < nb; ++e) {
                int ni = (int)((u >> bi[e]) & 1u) + (int)((d >> bi[e]) & 1u);
                int nj = (int)((u >> bj[e]) & 1u) + (int)((d >> bj[e]) & 1u);
                diag += V * (double)(ni * nj);
            }
            if (diag != 0.0) { rc[cnt] = (int32_t)(iu * Dd + id); rv[cnt] = diag; ++cnt; }
            /* hopping: -t c+_a c_b for every bond, both directions, both spins */
            for (int e = 0; e < nb; ++e) {
                for (int dir = 0; dir < 2; ++dir) {
                    const int a = dir ? bj[e] : bi[e];   /* created */
                    const int bsite = dir ? bi[e] : bj[e]; /* annihilated */
                    for (int spin = 0; spin < 2; ++spin) {
                        const int ma = a + spin * L, mb = bsite + spin * L;
                        if (!((occ >> mb) & 1u) || ((occ >> ma) & 1u)) continue;
                        int sgn = jw_sign_before(occ, mb);
                        uint64_t occ2 = occ & ~((uint64_t)1 << mb);
                        sgn *= jw_sign_before(occ2, ma);
                        occ2 |= (uint64_t)1 << ma;
                        const uint32_t u2 = (uint32_t)(occ2 & (full - 1));
                        const uint32_t d2 = (uint32_t)(occ2 >> L);
                        const int64_t j = (int64_t)rank_up[u2] * Dd + rank_dn[d2];
                        rc[cnt] = (int32_t)j; rv[cnt] = -t * (double)sgn; ++cnt;
                    }
                }
            }
            /* sort the row by column (insertion sort; rows are short) and merge duplicates */
            for (int x1 = 1; x1 < cnt; ++x1) {
                int32_t c0 = rc[x1]; double v0 = rv[x1]; int y = x1 - 1;
                while (y >= 0 && rc[y] > c0) { rc[y + 1] = rc[y]; rv[y + 1] = rv[y]; --y; }
                rc[y + 1] = c0; rv[y + 1] = v0;
            }
            int m = 0;
            for (int x1 = 0; x1 < cnt; ++x1) {
                if (m > 0 && rc[m - 1] == rc[x1]) rv[m - 1] += rv[x1];
                else { rc[m] = rc[x1]; rv[m] = rv[x1]; ++m; }
            }
            for (int x1 = 0; x1 < m; ++x1) {
                if (rv[x1] == 0.0) continue;
                if (col) { col[nnz] = rc[x1]; val[nnz] = rv[x1]; }
                ++nnz;
            }
            if (rowptr) rowptr[iu * Dd + id + 1] = nnz;
        }
    }
    (void)dim;
    free(rank); free(up_states); free(dn_states); free(rank_up); free(rank_dn); free(rc); free(rv);
    return nnz;
}

/* ------------------------------------------------------------------------ */
/* Two-orbital extended Hubbard model in a fixed (N_up, N_dn) sector: the
 * doubly degenerate model of Sec. IV.B (two orbitals per site, inter-site
 * Coulomb V), with the on-site interaction in the Kanamori form:
 *
 *   H = sum_{bonds (i,j)} sum_{a,b} sum_s t^{ij}_{ab} (c+_{ias} c_{jbs} + c+_{jbs} c_{ias})
 *     + U  sum_{i,a} n_{ia up} n_{ia dn}
 *     + U' sum_i n_{i0} n_{i1}                      (n_{ia} = n_{ia up} + n_{ia dn})
 *     - J  sum_i sum_s n_{i0s} n_{i1s}
 *     + J  sum_i sum_s c+_{i0s} c+_{i1s'} c_{i0s'} c_{i1s}   (s' = the other spin)
 *     + J' sum_i (c+_{i0 up} c+_{i0 dn} c_{i1 dn} c_{i1 up} + c+_{i1 up} c+_{i1 dn} c_{i0 dn} c_{i0 up})
 *     + V  sum_{bonds (i,j)} n_i n_j                 (n_i = n_{i0} + n_{i1})
 *
 * Modes: within a spin, mode 2 i + a (site i, orbital a); all up-spin modes
 * first, then all down-spin modes (offset 2 ns).  Every operator is applied
 * literally with its Jordan-Wigner sign (-1)^(occupied modes before it).
 * Basis: index = rank_up * D_dn + rank_dn, rank = position among the
 * (2 ns)-bit strings of the same popcount in ascending order (found by
 * enumeration).  t^{ij} is bond_t[b][a][b'] for bond b = (bond_i[b], bond_j[b]).
 * ------------------------------------------------------------------------ */
typedef struct {
    int ns, nb;
    const int32_t *bi, *bj;
    const double *bt;          /* [nb][2][2] */
    double U, Up, J, Jp, V;
    int n_up, n_dn;
    int64_t D_dn;
    const int32_t *rank;       /* [2^(2 ns)] rank among same-popcount strings */
} h2_model;

/* c_m (create = 0) or c+_m (create = 1) on occupation word *occ: returns the
 * Jordan-Wigner sign, or 0 when the operator annihilates the state. */
static int jw_apply(uint64_t *occ, int m, int create)
{
    const uint64_t bit = (uint64_t)1 << m;
    if (((*occ & bit) != 0) == (create != 0)) return 0;
    int c = 0;
    for (int j = 0; j < m; ++j) c += (int)((*occ >> j) & 1u);
    *occ ^= bit;
    return (c & 1) ? -1 : 1;
}

static int64_t h2_index(const h2_model *m, uint64_t occ)
{
    const int M = 2 * m->ns;
    const uint64_t mask = ((uint64_t)1 << M) - 1;
    return (int64_t)m->rank[occ & mask] * m->D_dn + m->rank[(occ >> M) & mask];
}

/* sequence of operators (rightmost applied first): ops[k] = mode, cre[k] = 1 for c+ */
static void h2_term(const h2_model *m, uint64_t occ, int nops, const int *ops, const int *cre, double coef,
                    int32_t *rc, double *rv, int *cnt)
{
    if (coef == 0.0) return;
    uint64_t o = occ;
    int sg = 1;
    for (int k = nops - 1; k >= 0; --k) {
        const int s = jw_apply(&o, ops[k], cre[k]);
        if (!s) return;
        sg *= s;
    }
    rc[*cnt] = (int32_t)h2_index(m, o);
    rv[*cnt] = coef * (double)sg;
    ++*cnt;
}

/* All terms of H applied to basis state occ: H|occ> = sum_k rv[k] |rc[k]>
 * (rc holds basis indices; duplicates not merged).  Returns the count. */
static int h2_apply_state(const h2_model *m, uint64_t occ, int32_t *rc, double *rv)
{
    const int M = 2 * m->ns;
    int cnt = 0;
    double diag = 0.0;
    for (int i = 0; i < m->ns; ++i) {
        int n[2][2];   /* n[a][s] */
        for (int a = 0; a < 2; ++a)
            for (int s = 0; s < 2; ++s) n[a][s] = (int)((occ >> (2 * i + a + s * M)) & 1u);
        diag += m->U * (double)(n[0][0] * n[0][1] + n[1][0] * n[1][1]);
        diag += m->Up * (double)((n[0][0] + n[0][1]) * (n[1][0] + n[1][1]));
        diag -= m->J * (double)(n[0][0] * n[1][0] + n[0][1] * n[1][1]);
    }
    for (int b = 0; b < m->nb; ++b) {
        int ni = 0, nj = 0;
        for (int a = 0; a < 2; ++a)
            for (int s = 0; s < 2; ++s) {
                ni += (int)((occ >> (2 * m->bi[b] + a + s * M)) & 1u);
                nj += (int)((occ >> (2 * m->bj[b] + a + s * M)) & 1u);
            }
        diag += m->V * (double)(ni * nj);
    }
    if (diag != 0.0) { rc[cnt] = (int32_t)h2_index(m, occ); rv[cnt] = diag; ++cnt; }
    /* hopping: t (c+_{i a s} c_{j b s} + c+_{j b s} c_{i a s}) */
    for (int b = 0; b < m->nb; ++b)
        for (int a = 0; a < 2; ++a)
            for (int a2 = 0; a2 < 2; ++a2) {
                const double t = m->bt[(size_t)b * 4 + a * 2 + a2];
                for (int s = 0; s < 2; ++s) {
                    const int mi = 2 * m->bi[b] + a + s * M, mj = 2 * m->bj[b] + a2 + s * M;
                    const int o1[2] = {mi, mj}, c1[2] = {1, 0};
                    const int o2[2] = {mj, mi}, c2[2] = {1, 0};
                    h2_term(m, occ, 2, o1, c1, t, rc, rv, &cnt);
                    h2_term(m, occ, 2, o2, c2, t, rc, rv, &cnt);
                }
            }
    /* spin flip and pair hopping on every site */
    for (int i = 0; i < m->ns; ++i) {
        for (int s = 0; s < 2; ++s) {
            const int so = 1 - s;
            const int ops[4] = {2 * i + 0 + s * M, 2 * i + 1 + so * M, 2 * i + 0 + so * M, 2 * i + 1 + s * M};
            const int cre[4] = {1, 1, 0, 0};
            h2_term(m, occ, 4, ops, cre, m->J, rc, rv, &cnt);
        }
        const int p1[4] = {2 * i + 0, 2 * i + 0 + M, 2 * i + 1 + M, 2 * i + 1};
        const int p2[4] = {2 * i + 1, 2 * i + 1 + M, 2 * i + 0 + M, 2 * i + 0};
        const int pc[4] = {1, 1, 0, 0};
        h2_term(m, occ, 4, p1, pc, m->Jp, rc, rv, &cnt);
        h2_term(m, occ, 4, p2, pc, m->Jp, rc, rv, &cnt);
    }
    return cnt;
}

static int h2_setup(h2_model *m, int ns, int nb, const int32_t *bi, const int32_t *bj, const double *bt,
                    double U, double Up, double J, double Jp, double V, int n_up, int n_dn,
                    int32_t **rank_out, uint32_t **up_out, uint32_t **dn_out, int64_t *Du, int64_t *Dd)
{
    if (ns < 1 || ns > 10 || nb < 0 || n_up < 0 || n_dn < 0 || n_up > 2 * ns || n_dn > 2 * ns) return -1;
    for (int b = 0; b < nb; ++b)
        if (bi[b] < 0 || bi[b] >= ns || bj[b] < 0 || bj[b] >= ns || bi[b] == bj[b]) return -1;
    const int M = 2 * ns;
    const uint32_t full = 1u << M;
    int32_t *rank = malloc(sizeof(int32_t) * full);
    uint32_t *up = malloc(sizeof(uint32_t) * full), *dn = malloc(sizeof(uint32_t) * full);
    if (!rank || !up || !dn) { free(rank); free(up); free(dn); return -3; }
    int64_t cu = 0, cd = 0, cnt[33] = {0};
    for (uint32_t s = 0; s < full; ++s) {
        const int p = popcount_u32(s);
        rank[s] = (int32_t)cnt[p]++;
        if (p == n_up) up[cu++] = s;
        if (p == n_dn) dn[cd++] = s;
    }
    m->ns = ns; m->nb = nb; m->bi = bi; m->bj = bj; m->bt = bt;
    m->U = U; m->Up = Up; m->J = J; m->Jp = Jp; m->V = V; m->n_up = n_up; m->n_dn = n_dn;
    m->D_dn = cd; m->rank = rank;
    *rank_out = rank; *up_out = up; *dn_out = dn; *Du = cu; *Dd = cd;
    return 0;
}

/* H of the sector in CSR (rows sorted by column, duplicates merged, exact
 * zeros dropped).  Call with rowptr/col/val NULL for the nnz (returned), then
 * with arrays of [dim+1], [nnz], [nnz]. */
int64_t oracle_hubbard2_csr(int ns, int nb, const int32_t *bi, const int32_t *bj, const double *bt,
                            double U, double Up, double J, double Jp, double V, int n_up, int n_dn,
                            int64_t *rowptr, int32_t *col, double *val)
{
    h2_model m;
    int32_t *rank; uint32_t *up, *dn; int64_t Du, Dd;
    int st = h2_setup(&m, ns, nb, bi, bj, bt, U, Up, J, Jp, V, n_up, n_dn, &rank, &up, &dn, &Du, &Dd);
    if (st) return st;
    const int cap = 1 + 16 * nb + 6 * ns;
    int32_t *rc = malloc(sizeof(int32_t) * cap);
    double *rv = malloc(sizeof(double) * cap);
    if (!rc || !rv) { free(rc); free(rv); free(rank); free(up); free(dn); return -3; }
    const int M = 2 * ns;
    int64_t nnz = 0;
    if (rowptr) rowptr[0] = 0;
    for (int64_t iu = 0; iu < Du; ++iu)
        for (int64_t id = 0; id < Dd; ++id) {
            const uint64_t occ = (uint64_t)up[iu] | ((uint64_t)dn[id] << M);
            int c = h2_apply_state(&m, occ, rc, rv);
            for (int x1 = 1; x1 < c; ++x1) {   /* insertion sort by column */
                int32_t c0 = rc[x1]; double v0 = rv[x1]; int y = x1 - 1;
                while (y >= 0 && rc[y] > c0) { rc[y + 1] = rc[y]; rv[y + 1] = rv[y]; --y; }
                rc[y + 1] = c0; rv[y + 1] = v0;
            }
            int k = 0;
            for (int x1 = 0; x1 < c; ++x1) {
                if (k > 0 && rc[k - 1] == rc[x1]) rv[k - 1] += rv[x1];
                else { rc[k] = rc[x1]; rv[k] = rv[x1]; ++k; }
            }
            for (int x1 = 0; x1 < k; ++x1) {
                if (rv[x1] == 0.0) continue;
                if (col) { col[nnz] = rc[x1]; val[nnz] = rv[x1]; }
                ++nnz;
            }
            if (rowptr) rowptr[iu * Dd + id + 1] = nnz;
        }
    free(rc); free(rv); free(rank); free(up); free(dn);
    return nnz;
}

/* y[r] = (H x)[rows[r]] for sampled rows of a sector too large for CSR: each
 * row from the terms of H applied to its basis state (H is real symmetric, so
 * row s holds the coefficients of H|s>).  x, y complex (re, im) pairs. */
int oracle_hubbard2_rows(int ns, int nb, const int32_t *bi, const int32_t *bj, const double *bt,
                         double U, double Up, double J, double Jp, double V, int n_up, int n_dn,
                         int64_t nrows, const int64_t *rows, const double *x, double *y)
{
    h2_model m;
    int32_t *rank; uint32_t *up, *dn; int64_t Du, Dd;
    int st = h2_setup(&m, ns, nb, bi, bj, bt, U, Up, J, Jp, V, n_up, n_dn, &rank, &up, &dn, &Du, &Dd);
    if (st) return st;
    const int M = 2 * ns;
    int bad = 0;
#pragma omp parallel
    {
        const int cap = 1 + 16 * nb + 6 * ns;
        int32_t *rc = malloc(sizeof(int32_t) * cap);
        double *rv = malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < nrows; ++r) {
            const int64_t s = rows[r];
            if (!rc || !rv || s < 0 || s >= Du * Dd) { bad = 1; continue; }
            const uint64_t occ = (uint64_t)up[s / Dd] | ((uint64_t)dn[s % Dd] << M);
            const int c = h2_apply_state(&m, occ, rc, rv);
            double re = 0.0, im = 0.0;
            for (int k = 0; k < c; ++k) { re += rv[k] * x[2 * (size_t)rc[k]]; im += rv[k] * x[2 * (size_t)rc[k] + 1]; }
            y[2 * r] = re; y[2 * r + 1] = im;
        }
        free(rc); free(rv);
    }
    free(rank); free(up); free(dn);
    return bad ? -1 : 0;
}
