"""Pins for the CPU oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: dense LU,
closed forms, invariants of the method (collinear residuals, seed
independence), a Fock-space construction of the Hubbard model, numbers the
paper prints.  A dropped term, a wrong sign or a transposed operand anywhere in
the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_0802_0748_gb300 import inputs
from oracle import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def relerr(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def small_anderson(L=3, seed=11):
    return inputs.anderson_csr(L, seed=seed)


# ---------------------------------------------------------------- apply
def test_apply_matches_scipy(oracle_mod):
    h = small_anderson()
    x = inputs.random_unit_complex(h.n, 7)
    z = 0.3 + 0.02j
    y = oracle_mod.apply_shifted(h.rowptr, h.col, h.val, z, x)
    ref = z * x - h.scipy() @ x
    assert np.allclose(y, ref, rtol=0, atol=1e-14)


# ---------------------------------------------------------------- dense LU
@pytest.mark.parametrize("seed_rule", [-1, 0, 4])
def test_shifted_cocg_matches_dense_lu(oracle_mod, seed_rule):
    """G_mk = c_m^T (z_k - H)^{-1} b (Eq. gf) against dense LU, several seeds."""
    h = small_anderson()
    b = inputs.random_unit_complex(h.n, 3)
    C = np.stack([np.conj(b), inputs.random_unit_complex(h.n, 4)])
    shifts = np.linspace(-4.0, 4.0, 9) + 0.05j
    res = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_vec=C, tol=1e-13,
                                  seed=seed_rule)
    assert res.status == oracle_mod.OK
    ref = dense.green_dense(h.dense(), shifts, b, C)
    assert relerr(res.G, ref) < 1e-10


def test_unit_projections_and_complex_shift_spread(oracle_mod):
    """Projections e_i and shifts with different imaginary parts (sigma complex)."""
    h = small_anderson(seed=12)
    b = inputs.random_unit_complex(h.n, 5)
    idx = np.array([0, 17, h.n - 1])
    shifts = np.array([-1.0 + 0.02j, 0.5 + 0.1j, 2.0 + 0.5j, -3.0 + 0.05j])
    res = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_idx=idx, tol=1e-13)
    assert res.status == oracle_mod.OK
    C = np.zeros((3, h.n), dtype=complex); C[np.arange(3), idx] = 1.0
    ref = dense.green_dense(h.dense(), shifts, b, C)
    assert relerr(res.G, ref) < 1e-10
    # seed rule: smallest Im z is shift 0
    assert oracle_mod.default_seed(shifts) == 0


# ---------------------------------------------------------------- closed forms
def test_chain_exact_closed_form(oracle_mod):
    """Open chain (t=-1): G_00 equals the exact finite-chain eigen-sum."""
    L = 256
    h = inputs.chain_csr(L, t=-1.0)
    shifts = np.linspace(-2.5, 2.5, 64) + 0.01j
    b = np.zeros(L, complex); b[0] = 1
    res = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_idx=[0], tol=1e-13)
    assert res.status == oracle_mod.OK
    ref = dense.chain_g00_exact(L, -1.0, shifts)
    assert relerr(res.G[0], ref) < 1e-10


def test_chain_closed_forms_agree():
    """The finite-chain sum reaches the surface form at L=4096 and the bulk form mid-chain."""
    z = np.linspace(-2.5, 2.5, 64) + 0.01j
    g_exact = dense.chain_g00_exact(4096, -1.0, z)
    g_surf = dense.chain_g00_surface(-1.0, z)
    assert np.max(np.abs(g_exact - g_surf)) < 1e-12
    # bulk: centre site of a long chain, dense diagonalisation
    L = 1201
    H = inputs.chain_csr(L, t=-1.0).dense()
    w, U = np.linalg.eigh(H)
    j = L // 2
    zz = np.array([-1.0 + 0.05j, 0.3 + 0.05j, 1.7 + 0.05j])
    g_mid = (U[j, :] ** 2 / (zz[:, None] - w[None, :])).sum(axis=1)
    assert np.max(np.abs(g_mid - dense.chain_gjj_bulk(-1.0, zz))) < 1e-6


def test_chain_surface_form_is_semi_infinite_limit():
    """Surface form satisfies g = 1/(z - t^2 g) (one site attached to a semi-infinite chain)."""
    z = np.linspace(-3, 3, 41) + 0.01j
    g = dense.chain_g00_surface(-1.0, z)
    assert np.max(np.abs(g - 1.0 / (z - g))) < 1e-12
    assert np.all(g.imag < 0)


# ---------------------------------------------------------------- invariants
def test_collinear_residuals(oracle_mod):
    """True residual b - (z_k - H) x^k_n equals r_n / pi^k_n (collinear residuals, Sec. III.C)."""
    h = small_anderson(L=4, seed=13)
    b = inputs.random_unit_complex(h.n, 6)
    shifts = np.linspace(-3.0, 3.0, 7) + 0.1j
    for nit in (1, 2, 10, 40):
        res = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_idx=[0], tol=0.0,
                                      max_iter=nit, want_x=True, want_state=True)
        assert res.status == oracle_mod.NOT_CONVERGED and res.n_iter == nit
        for k, z in enumerate(shifts):
            true_r = b - oracle_mod.apply_shifted(h.rowptr, h.col, h.val, z, res.X[k])
            rec_r = res.r / res.pi[k]
            assert np.linalg.norm(true_r - rec_r) <= 1e-11 * max(np.linalg.norm(true_r), 1e-3)


def test_sigma_zero_pi_is_one(oracle_mod):
    """A shift equal to the seed has sigma = 0 and pi identically 1."""
    h = small_anderson(L=3, seed=14)
    b = inputs.random_unit_complex(h.n, 8)
    shifts = np.array([0.2 + 0.01j, 1.0 + 0.05j, 0.2 + 0.01j])
    res = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_idx=[1], tol=0.0,
                                  max_iter=25, seed=0, want_state=True)
    assert res.pi[0] == 1.0 and res.pi[2] == 1.0
    assert res.G[0, 0] == res.G[0, 2]


def test_first_iterate_closed_form(oracle_mod):
    """After one step, x^k_1 = alpha^k_0 b with alpha^k_0 = (b^T b)/(b^T (z_k - H) b)."""
    h = small_anderson(L=3, seed=15)
    b = inputs.random_unit_complex(h.n, 9)
    shifts = np.array([0.3 + 0.05j, -1.2 + 0.2j])
    res = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_vec=[b], tol=0.0,
                                  max_iter=1, want_x=True)
    for k, z in enumerate(shifts):
        Ab = z * b - h.scipy() @ b
        a = (b @ b) / (b @ Ab)
        assert np.allclose(res.X[k], a * b, rtol=1e-13, atol=1e-15)


def test_shift_iterates_equal_plain_cocg_per_shift(oracle_mod):
    """The shifted iterate x^k_n equals COCG run directly on shift k (Eq. inv_KS):
    running with the seed at z_k gives the same x^k_n at the same n."""
    h = small_anderson(L=3, seed=16)
    b = inputs.random_unit_complex(h.n, 10)
    shifts = np.array([-0.5 + 0.05j, 0.7 + 0.05j, 2.0 + 0.3j])
    n = 15
    a = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_idx=[0], tol=0.0,
                                max_iter=n, seed=0, want_x=True)
    for k in range(3):
        d = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts[k:k + 1], b, proj_idx=[0],
                                    tol=0.0, max_iter=n, seed=0, want_x=True)
        assert np.linalg.norm(a.X[k] - d.X[0]) < 1e-9 * np.linalg.norm(d.X[0])


def test_seed_switching_keeps_result(oracle_mod):
    """A seed that converges first forces switches; results stay those of dense LU."""
    h = small_anderson(L=4, seed=17)
    b = inputs.random_unit_complex(h.n, 11)
    shifts = np.concatenate([[30.0 + 1.0j], np.linspace(-3, 3, 6) + 0.02j, [-25.0 + 0.5j]])
    res = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_vec=[np.conj(b)],
                                  tol=1e-12, seed=0)
    assert res.status == oracle_mod.OK
    assert res.n_switch >= 1 and res.seed != 0
    ref = dense.green_dense(h.dense(), shifts, b, [np.conj(b)])
    assert relerr(res.G, ref) < 1e-9
    no_switch = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_vec=[np.conj(b)],
                                        tol=1e-12, seed=0, allow_switch=False)
    assert no_switch.status == oracle_mod.ERR_BREAKDOWN


def test_residual_monitor_bounds_error(oracle_mod):
    """|G - G_exact| <= ||c|| ||(z-H)^{-1}|| ||r|| <= ||c|| ||b|| tol / Im z (Eq. residual)."""
    h = small_anderson(L=3, seed=18)
    b = inputs.random_unit_complex(h.n, 12)
    shifts = np.linspace(-4, 4, 11) + 0.03j
    tol = 1e-6
    res = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_vec=[np.conj(b)], tol=tol)
    ref = dense.green_dense(h.dense(), shifts, b, [np.conj(b)])
    assert np.all(res.resid <= tol)
    assert np.all(np.abs(res.G - ref)[0] <= tol / shifts.imag * 1.0001)


def test_dos_sum_rule(oracle_mod):
    """-(1/pi) int Im G_jj(E + i eta) dE = 1: trapezoid over [-W, W] plus the Lorentzian tail."""
    L = 48
    h = inputs.chain_csr(L, t=-1.0)
    eta, W = 0.05, 8.0
    E = np.linspace(-W, W, 6401)
    b = np.zeros(L, complex); b[L // 3] = 1
    res = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, E + 1j * eta, b, proj_idx=[L // 3],
                                  tol=1e-12)
    dos = -res.G[0].imag / np.pi
    integral = np.trapezoid(dos, E)
    tail = 1.0 - (2.0 / np.pi) * math.atan(W / eta)
    assert abs(integral + tail - 1.0) < 2e-3
    assert np.all(dos > 0)


def test_stopping_and_breakdown_edges(oracle_mod):
    h = small_anderson(L=3, seed=19)
    b = np.zeros(h.n, complex)
    res = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, [0.1 + 0.1j], b, proj_idx=[0])
    assert res.status == oracle_mod.OK and res.G[0, 0] == 0
    b = inputs.random_unit_complex(h.n, 1)
    res = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, [0.1 + 0.001j], b, proj_idx=[0],
                                  tol=1e-14, max_iter=3)
    assert res.status == oracle_mod.NOT_CONVERGED and res.n_iter == 3


# ---------------------------------------------------------------- Hubbard
def test_paper_sector_dimension(oracle_mod):
    """(16 C 6)^2 = 64,128,064 (Sec. IV.B) and (14 C 7)^2 = 11,778,624 by enumeration."""
    g = json.load(open(os.path.join(GOLDEN, "paper_numbers.json")))["hubbard_sector_dim"]
    d = oracle_mod.sector_dim(g["modes_per_spin"], g["electrons_per_spin"])
    assert d * d == g["value"] == 64128064
    assert oracle_mod.sector_dim(14, 7) ** 2 == 11778624


@pytest.mark.parametrize("L,nu,nd,periodic", [(2, 1, 1, True), (3, 1, 2, True), (4, 2, 2, True),
                                              (4, 1, 2, False), (5, 2, 3, True)])
def test_hubbard_csr_equals_fock_construction(oracle_mod, L, nu, nd, periodic):
    t, U, V = 1.0, 4.0, 1.0
    rp, c, v = oracle_mod.hubbard_csr(L, nu, nd, t, U, V, periodic)
    n = rp.size - 1
    import scipy.sparse as sp
    Hc = sp.csr_matrix((v, c, rp), shape=(n, n)).toarray()
    Hf = dense.fock_hubbard_sector(L, nu, nd, t, U, V, periodic)
    assert np.array_equal(Hc, Hf)
    assert np.array_equal(Hc, Hc.T)


def test_two_site_hubbard_spectrum(oracle_mod):
    rp, c, v = oracle_mod.hubbard_csr(2, 1, 1, 1.0, 4.0, 1.0, True)
    import scipy.sparse as sp
    H = sp.csr_matrix((v, c, rp), shape=(4, 4)).toarray()
    w = np.linalg.eigvalsh(H)
    assert np.allclose(w, dense.two_site_spectrum(1.0, 4.0, 1.0), atol=1e-13)
    assert np.allclose(w, [0, 1, 4, 5], atol=1e-13)


def test_four_site_free_fermions_periodic(oracle_mod):
    rp, c, v = oracle_mod.hubbard_csr(4, 2, 2, 1.0, 0.0, 0.0, True)
    import scipy.sparse as sp
    H = sp.csr_matrix((v, c, rp), shape=(36, 36)).toarray()
    assert np.allclose(np.linalg.eigvalsh(H), dense.free_fermion_sector_spectrum(4, 2, 2, 1.0),
                       atol=1e-12)


def test_hubbard_green_function_dense(oracle_mod):
    """Shifted COCG on a 4-site Hubbard sector against dense LU of the Fock construction."""
    H = dense.fock_hubbard_sector(4, 2, 2, 1.0, 4.0, 1.0, True)
    rp, c, v = oracle_mod.hubbard_csr(4, 2, 2, 1.0, 4.0, 1.0, True)
    b = inputs.random_unit_complex(36, 21)
    shifts = np.linspace(-6, 12, 10) + 0.05j
    res = oracle_mod.shifted_cocg(rp, c, v, shifts, b, proj_vec=[np.conj(b)], tol=1e-13)
    ref = dense.green_dense(H, shifts, b, [np.conj(b)])
    assert relerr(res.G, ref) < 1e-10


# ---------------------------------------------------------------- gradient
def test_dense_gradient_matches_finite_difference():
    """grad_dense against central differences of dense LU on a symmetric pair (a, b), (b, a)."""
    h = small_anderson(L=3, seed=22)
    H = h.dense()
    n = H.shape[0]
    b = np.zeros(n, complex); b[0] = 1
    shifts = np.linspace(-3, 3, 5) + 0.1j
    w = np.random.default_rng(0).normal(size=5)
    gbar = 1j * w
    g = dense.grad_dense(H, shifts, b, b, gbar)

    def loss(Hm):
        return float(np.sum(w * dense.green_dense(Hm, shifts, b, [b])[0].imag))
    for (a, c) in [(0, 0), (0, 1), (5, 9), (17, 40)]:
        E = np.zeros_like(H); E[a, c] += 1; E[c, a] += 1 if a != c else 0
        step = 1e-5
        fd = (loss(H + step * E) - loss(H - step * E)) / (2 * step)
        an = g[a, c] + (g[c, a] if a != c else 0)
        assert abs(fd - an) < 1e-7 * max(1.0, abs(an))


def test_iterates_after_switch_equal_plain_cocg(oracle_mod):
    """After a seed switch the iterates of the remaining shifts are still those
    of COCG run directly on each shift (Eq. inv_KS: one Krylov space serves all)."""
    h = small_anderson(L=3, seed=23)
    b = inputs.random_unit_complex(h.n, 13)
    shifts = np.array([40.0 + 2.0j, -0.4 + 0.05j, 0.9 + 0.05j, 2.5 + 0.1j])
    n = 30
    a = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_idx=[0], tol=1e-9,
                                max_iter=n, seed=0, want_x=True)
    assert a.n_switch >= 1 and a.n_iter == n and a.iters[0] < n
    for k in range(1, 4):
        if a.iters[k] < n:
            continue
        d = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts[k:k + 1], b, proj_idx=[0],
                                    tol=0.0, max_iter=n, seed=0, want_x=True)
        assert np.linalg.norm(a.X[k] - d.X[0]) < 1e-9 * np.linalg.norm(d.X[0])


def test_fixed_iterates_are_seed_independent_before_ritz_convergence(oracle_mod):
    """Early iterates do not depend on the seed (same Krylov space, Eq. inv_KS)."""
    h = small_anderson(L=6, seed=5)
    b = inputs.random_unit_complex(h.n, 9)
    shifts = np.linspace(-5, 5, 12) + 0.05j
    a = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_vec=[np.conj(b)], tol=0.0,
                                max_iter=20, seed=3)
    c = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_vec=[np.conj(b)], tol=0.0,
                                max_iter=20, seed=8)
    assert relerr(a.G, c.G) < 1e-10


# ------------------------------------------------------------------ density matrix (Eq. densityM)
def test_density_half_filling_bipartite_is_one_half():
    """Closed form: on a bipartite lattice with zero onsite energy the spectrum is
    symmetric and every site holds exactly 1/2 at mu = 0, at any temperature
    (an even chain: no zero mode on the step of the kT = 0 occupation)."""
    from oracle import dense
    L = 16
    H = np.diag(-np.ones(L - 1), 1) + np.diag(-np.ones(L - 1), -1)
    for kT in (0.0, 0.05, 0.7):
        for j in (0, 5, 15):
            e = np.zeros(L); e[j] = 1.0
            assert abs(dense.density_exact(H, e, [e], 0.0, kT)[0] - 0.5) < 1e-13


def test_density_limits_count_and_completeness():
    """kT = 0: the trace is the number of eigenvalues below mu; mu far above the
    spectrum: rho = c^T b (completeness of the eigenvectors)."""
    from oracle import dense
    rng = np.random.default_rng(5)
    A = rng.normal(size=(12, 12)); H = (A + A.T) / 2
    lam = np.linalg.eigvalsh(H)
    mu = 0.5 * (lam[4] + lam[5])
    I = np.eye(12)
    tr = sum(dense.density_exact(H, I[j], [I[j]], mu, 0.0)[0] for j in range(12))
    assert abs(tr - 5.0) < 1e-12
    b = rng.normal(size=12) + 1j * rng.normal(size=12)
    c = rng.normal(size=12)
    assert abs(dense.density_exact(H, b, [c], 1e3, 0.1)[0] - c @ b) < 1e-12


def test_density_quadrature_converges_to_eigenstate_sum():
    """Eq. densityM on a broadened real-axis grid approaches the Fermi-weighted
    eigenstate sum (Eq. densityM-1) as delta -> 0: the error of the Lorentzian
    smoothing of f is O(delta / kT), so halving delta roughly halves it."""
    from oracle import dense
    rng = np.random.default_rng(9)
    A = rng.normal(size=(16, 16)); H = (A + A.T) / 4
    lo, hi = np.linalg.eigvalsh(H)[[0, -1]]
    e0 = np.eye(16)[0]
    mu, kT = 0.1, 0.2
    exact = dense.density_exact(H, e0, [e0], mu, kT)[0]
    errs = []
    for delta in (0.04, 0.02, 0.01):
        grid = np.linspace(lo - 4.0, hi + 4.0, int(round((hi - lo + 8.0) / (delta / 8))) + 1)
        G = dense.green_dense(H, grid + 1j * delta, e0, [e0])
        errs.append(abs(dense.density_quadrature(G, grid, mu, kT)[0] - exact))
    assert errs[2] < 0.65 * errs[1] < 0.65 ** 2 * errs[0]
    assert errs[2] < 1e-2


def test_vector_gradient_equals_dense_gradient(oracle_mod):
    """The gradient from the oracle's full shifted-COCG solutions (forward with b,
    adjoint with c) equals the dense-inverse gradient on every stored entry;
    with c = b the adjoint solutions are the forward ones."""
    h = inputs.anderson_csr(3, seed=8)
    n = h.n
    shifts = np.linspace(-4, 4, 9) + 0.07j
    b = inputs.random_unit_complex(n, 3)
    c = inputs.random_unit_complex(n, 4)
    gbar = np.random.default_rng(5).normal(size=9) + 1j * np.random.default_rng(6).normal(size=9)
    X = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, b, proj_idx=[0], tol=1e-14, want_x=True).X
    Y = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts, c, proj_idx=[0], tol=1e-14, want_x=True).X
    rows = np.repeat(np.arange(n), np.diff(h.rowptr))
    for yy, cc in ((Y, c), (X, b)):
        g = oracle_mod.grad_from_vectors(h.rowptr, h.col, X, yy, gbar)
        ref = dense.grad_dense(h.dense(), shifts, b, cc, gbar)[rows, h.col]
        assert np.max(np.abs(g - ref)) < 1e-10 * np.max(np.abs(ref))
    # a transposed operand (x_k[a] y_k[b]) is a different gradient when c != b
    gt = oracle_mod.grad_from_vectors(h.rowptr, h.col, Y, X, gbar)
    ref = dense.grad_dense(h.dense(), shifts, b, c, gbar)[rows, h.col]
    assert np.max(np.abs(gt - ref)) > 1e-3 * np.max(np.abs(ref))


# ---------------------------------------------------------------- two-orbital model (Sec. IV.B)
def _model2(bonds, dirs, seed=None, **over):
    m = inputs.eg_model(bonds=bonds, dirs=dirs, **over)
    if seed is not None:   # generic hoppings: no accidental symmetry hides a wrong sign or index
        rng = np.random.default_rng(seed)
        m["bond_t"] = rng.normal(size=(len(bonds), 2, 2)).tolist()
    return m


@pytest.mark.parametrize("nu,nd", [(1, 1), (2, 1), (2, 2), (3, 1), (1, 3)])
def test_hubbard2_csr_equals_fock_construction(oracle_mod, nu, nd):
    """Two sites, one bond, generic hoppings and interaction values: the sector
    CSR built term by term from bit strings equals the Fock-space Kronecker
    construction restricted to the sector."""
    m = _model2([(0, 1)], [0], seed=3, U=3.1, Up=1.7, J=0.6, Jp=0.45, V=0.8)
    Hf, _, _ = dense.fock_hubbard2(m)
    ref = dense.fock_sector2(Hf, 2, nu, nd)
    rp, c, v = oracle_mod.hubbard2_csr(m, nu, nd)
    n = rp.size - 1
    import scipy.sparse as sp
    H = sp.csr_matrix((v, c, rp), shape=(n, n)).toarray()
    assert np.max(np.abs(H - ref)) < 1e-13
    assert np.max(np.abs(H - H.T)) == 0.0


def test_hubbard2_atomic_kanamori_levels(oracle_mod):
    """One site: the S_z = 0 two-electron levels are U' -+ J and U -+ J'; the
    S_z = 1 state sits at U' - J (the same triplet)."""
    m = {"n_sites": 1, "bonds": [], "bond_t": np.zeros((0, 2, 2)), "U": 4.0, "Up": 2.5, "J": 0.75, "Jp": 0.6,
         "V": 1.0}
    rp, c, v = oracle_mod.hubbard2_csr(m, 1, 1)
    import scipy.sparse as sp
    H = sp.csr_matrix((v, c, rp), shape=(4, 4)).toarray()
    assert np.allclose(np.linalg.eigvalsh(H), dense.kanamori_two_electron_levels(4.0, 2.5, 0.75, 0.6), atol=1e-14)
    rp2, c2, v2 = oracle_mod.hubbard2_csr(m, 2, 0)
    assert rp2.size == 2 and np.allclose(v2, [2.5 - 0.75])


def test_hubbard2_fock_model_is_spin_invariant():
    """With U' = U - 2J and J' = J the Kanamori interaction is spin-rotation
    invariant: H commutes with S^2 and S_z (a wrong sign of the spin-flip or
    pair-hopping term breaks [H, S^2] = 0)."""
    m = _model2([(0, 1)], [0], seed=5, U=3.0, Up=1.8, J=0.6, Jp=0.6, V=0.7)
    H, c, _ = dense.fock_hubbard2(m)
    S2, Sz = dense.fock_spin2(2, c)
    assert np.max(np.abs(H @ S2 - S2 @ H)) < 1e-12
    assert np.max(np.abs(H @ Sz - Sz @ H)) < 1e-12
    # the same H with the spin-flip term (alone) of the opposite sign is not
    cd = [x.T for x in c]
    sf = sum(cd[2 * i + 0 + 4 * s] @ cd[2 * i + 1 + 4 * (1 - s)] @ c[2 * i + 0 + 4 * (1 - s)] @ c[2 * i + 1 + 4 * s]
             for i in range(2) for s in range(2))
    Hb = H - 2 * 0.6 * sf
    assert np.max(np.abs(Hb @ S2 - S2 @ Hb)) > 1e-3


def test_hubbard2_free_fermions_on_sqrt8_cluster(oracle_mod):
    """Hopping alone on the sqrt(8) x sqrt(8) cluster: the sector spectrum is
    every sum of occupied single-particle energies (2 up, 1 down)."""
    m = inputs.eg_model(U=0.0, Up=0.0, J=0.0, Jp=0.0, V=0.0)
    rp, c, v = oracle_mod.hubbard2_csr(m, 2, 1)
    import scipy.sparse as sp
    n = rp.size - 1
    ev = np.linalg.eigvalsh(sp.csr_matrix((v, c, rp), shape=(n, n)).toarray())
    assert np.allclose(ev, dense.free_fermion_spectrum2(m, 2, 1), atol=1e-12)


def test_hubbard2_rows_equal_csr_product(oracle_mod):
    """Sampled rows of H x computed state by state equal the CSR product
    (sqrt(8) x sqrt(8), 2 up 2 down, 14,400 states); the 6/6 sector of the
    paper has (16 C 6)^2 states."""
    m = inputs.eg_model()
    rp, c, v = oracle_mod.hubbard2_csr(m, 2, 2)
    n = rp.size - 1
    assert n == math.comb(16, 2) ** 2
    x = inputs.random_unit_complex(n, 9)
    import scipy.sparse as sp
    y = sp.csr_matrix((v, c, rp), shape=(n, n)) @ x
    rows = np.random.default_rng(1).choice(n, 300, replace=False)
    assert np.max(np.abs(oracle_mod.hubbard2_rows(m, 2, 2, rows, x) - y[rows])) < 1e-14
    assert oracle_mod.sector_dim(16, 6) ** 2 == 64128064
