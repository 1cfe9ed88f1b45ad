"""Pins for the ground-state and excitation part of the oracle (Sec. II.B,
Sec. IV.B) against what the mathematics fixes: dense eigen-decomposition,
closed forms (free fermions on a ring, two sites), the canonical
anticommutation relations, the Kronecker-product construction of the
Jordan-Wigner operators, sum rules and the high-energy expansion of G.  A
dropped beta term or a wrong sign in the Lanczos, CG or operator code fails
at least one of them.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import dense, ground
from paper_0802_0748_gb300 import inputs


def hubbard(oracle_mod, L, nu, nd, t=1.0, U=4.0, V=1.0, periodic=True):
    rowptr, col, val = oracle_mod.hubbard_csr(L, nu, nd, t, U, V, periodic)
    n = rowptr.size - 1
    return sp.csr_matrix((val, col, rowptr), shape=(n, n))


def exact_ground(H):
    E, U = np.linalg.eigh(H.toarray() if sp.issparse(H) else H)
    return E, U


@pytest.mark.parametrize("m,cg", [(20, 0), (20, 40), (60, 0)])
def test_lanczos_cycle_matches_dense_eigh(oracle_mod, m, cg):
    """Hubbard ring L=6, 3 up 3 down (400 states): E to 1e-10, psi up to sign."""
    H = hubbard(oracle_mod, 6, 3, 3)
    E, U = exact_ground(H)
    assert E[1] - E[0] > 1e-2            # a unique ground state
    gs = ground.lanczos_ground_state(H, inputs.random_unit_real(H.shape[0], 1), m=m, cg_steps=cg, tol=1e-10)
    assert gs.status == 0 and gs.resid <= 1e-10
    assert abs(gs.energy - E[0]) < 1e-10
    assert abs(abs(gs.psi @ U[:, 0]) - 1.0) < 1e-12


def test_lanczos_free_fermions_closed_form(oracle_mod):
    """U = V = 0 on a ring with an odd number of electrons per spin (closed
    shell): E_0 = sum of the lowest -2 t cos(2 pi m / L)."""
    H = hubbard(oracle_mod, 10, 5, 5, U=0.0, V=0.0)
    gs = ground.lanczos_ground_state(H, inputs.random_unit_real(H.shape[0], 2), m=60, tol=1e-9)
    assert gs.status == 0
    assert abs(gs.energy - ground.free_fermion_ground_energy(10, 5, 5, 1.0)) < 1e-10


def test_lanczos_two_sites_closed_form_and_early_stop(oracle_mod):
    """Two sites, one bond, one electron per spin (4 states): the Lanczos
    recursion stops at the invariant subspace before m steps and E_0 =
    (U+V)/2 - sqrt(((U-V)/2)^2 + 4 t^2)."""
    H = hubbard(oracle_mod, 2, 1, 1, U=3.0, V=0.5, periodic=False)
    gs = ground.lanczos_ground_state(H, inputs.random_unit_real(4, 3), m=10, tol=1e-12)
    assert gs.status == 0 and gs.lanczos_steps <= 4
    assert abs(gs.energy - dense.two_site_spectrum(1.0, 3.0, 0.5)[0]) < 1e-13


def test_lanczos_start_at_eigenvector(oracle_mod):
    """Started at the ground state, one Lanczos step spans an invariant
    subspace (beta_0 = 0 to rounding) and the first cycle converges."""
    H = hubbard(oracle_mod, 6, 3, 3)
    E, U = exact_ground(H)
    gs = ground.lanczos_ground_state(H, U[:, 0], m=30, tol=1e-11)
    assert gs.status == 0 and gs.cycles == 1 and gs.lanczos_steps == 1
    assert abs(gs.energy - E[0]) < 1e-12


def test_cg_inverse_step_contracts_excited_component(oracle_mod):
    """One CG inverse-iteration solve with sigma below E_0 multiplies the
    excited-state admixture by (E_0 - sigma) / (E_1 - sigma) (exact solve)."""
    H = hubbard(oracle_mod, 6, 3, 3)
    E, U = exact_ground(H)
    psi = U[:, 0] + 0.3 * U[:, 1]
    psi /= np.linalg.norm(psi)
    sigma = E[0] - 0.05
    y = ground._cg_inverse_step(H, psi, sigma, 400)
    ratio = (y @ U[:, 1]) / (y @ U[:, 0])
    assert abs(ratio / 0.3 - (E[0] - sigma) / (E[1] - sigma)) < 1e-6


def test_cg_not_run_on_indefinite_shift(oracle_mod):
    """p^T (H - sigma) p <= 0 at the first step: the CG solve returns y = 0."""
    H = hubbard(oracle_mod, 4, 2, 2)
    psi = inputs.random_unit_real(H.shape[0], 5)
    y = ground._cg_inverse_step(H, psi, float(psi @ (H @ psi)) + 100.0, 10)
    assert np.all(y == 0)


# ------------------------------------------------------------ fermion operators
def kron_sector_index(L, nu, nd):
    """Kronecker-basis indices (mode 0 most significant) of a sector's states in
    the rank order used by the solver."""
    M = 2 * L
    ups, dns = dense.sector_states(L, nu), dense.sector_states(L, nd)
    idx = []
    for u in ups:
        for d in dns:
            bits = [(u >> i) & 1 for i in range(L)] + [(d >> i) & 1 for i in range(L)]
            idx.append(sum(bits[m] << (M - 1 - m) for m in range(M)))
    return np.array(idx)


@pytest.mark.parametrize("create", [False, True])
def test_fermion_op_equals_kronecker_construction(create):
    """c_m (and c+_m) between sectors equal the Jordan-Wigner Kronecker
    products Z x ... x Z x a x 1 x ... restricted to the sectors (L = 3)."""
    L, nu, nd = 3, 2, 1
    c = dense._jw_annihilators(2 * L)
    src = kron_sector_index(L, nu, nd)
    psi = inputs.random_unit_real(src.size, 7)
    for site, spin in itertools.product(range(L), range(2)):
        d = 1 if create else -1
        tu, td = (nu + d, nd) if spin == 0 else (nu, nd + d)
        if not (0 <= tu <= L and 0 <= td <= L):
            continue
        op = c[site + spin * L].T if create else c[site + spin * L]
        dst = kron_sector_index(L, tu, td)
        ref = op[np.ix_(dst, src)] @ psi
        got = ground.fermion_op(L, nu, nd, site, spin, create, psi)
        assert np.array_equal(got, ref), (site, spin)


def test_fermion_op_anticommutation():
    """{c_a, c+_b} = delta_ab and {c_a, c_b} = 0 on random sector vectors (L = 4)."""
    L, nu, nd = 4, 2, 1
    psi = inputs.random_unit_real(6 * 4, 8)
    modes = [(s, p) for p in range(2) for s in range(L)]
    for (i, si), (j, sj) in itertools.product(modes, modes):
        # c_i c+_j psi + c+_j c_i psi
        up1 = (nu + (sj == 0), nd + (sj == 1))
        a = ground.fermion_op(L, *up1, i, si, False, ground.fermion_op(L, nu, nd, j, sj, True, psi))
        dn1 = (nu - (si == 0), nd - (si == 1))
        b = ground.fermion_op(L, *dn1, j, sj, True, ground.fermion_op(L, nu, nd, i, si, False, psi))
        assert np.allclose(a + b, psi if (i, si) == (j, sj) else 0.0, atol=1e-15)
        if (i, si) != (j, sj):
            # c_i c_j psi + c_j c_i psi = 0
            dj = (nu - (sj == 0), nd - (sj == 1))
            x = ground.fermion_op(L, *dj, i, si, False, ground.fermion_op(L, nu, nd, j, sj, False, psi)) \
                if min(dj[0] - (si == 0), dj[1] - (si == 1)) >= 0 else 0.0
            y = ground.fermion_op(L, *dn1, j, sj, False, ground.fermion_op(L, nu, nd, i, si, False, psi)) \
                if min(dn1[0] - (sj == 0), dn1[1] - (sj == 1)) >= 0 else 0.0
            assert np.allclose(np.asarray(x) + np.asarray(y), 0.0, atol=1e-15)


def test_number_operator_and_occupations():
    """c+_i c_i is diagonal with the occupation of mode i; its expectation is
    ground.occupations."""
    L, nu, nd = 4, 2, 2
    psi = inputs.random_unit_real(36, 9)
    occ = ground.occupations(L, nu, nd, psi)
    for i, s in itertools.product(range(L), range(2)):
        tgt = (nu - (s == 0), nd - (s == 1))
        np_ = ground.fermion_op(L, *tgt, i, s, True, ground.fermion_op(L, nu, nd, i, s, False, psi))
        assert abs(psi @ np_ - occ[s, i]) < 1e-14
    assert np.allclose(occ.sum(axis=1), [nu, nd], atol=1e-13)


def test_ground_state_occupation_sum_rule(oracle_mod):
    """Translation-invariant unique ground state on the ring: ||c_{i s} psi_0||^2
    = <n_{i s}> = N_s / L for every site."""
    L, nu, nd = 6, 3, 3
    H = hubbard(oracle_mod, L, nu, nd)
    gs = ground.lanczos_ground_state(H, inputs.random_unit_real(H.shape[0], 4), m=40, tol=1e-11)
    for i in range(L):
        b = ground.fermion_op(L, nu, nd, i, 0, False, gs.psi)
        assert abs(b @ b - nu / L) < 1e-10


def test_excitation_green_lehmann_and_moments(oracle_mod):
    """G(z) = b^T (z - H)^{-1} b for the ionization vector b = c_{0 up} psi_0:
    dense solves equal the Lehmann sum, and at large |z| G -> |b|^2 / z +
    b^T H b / z^2."""
    L, nu, nd = 6, 3, 3
    H = hubbard(oracle_mod, L, nu, nd)
    gs = ground.lanczos_ground_state(H, inputs.random_unit_real(H.shape[0], 4), m=40, tol=1e-11)
    b = ground.fermion_op(L, nu, nd, 0, 0, False, gs.psi)
    Hm = hubbard(oracle_mod, L, nu - 1, nd)
    z = gs.energy - np.linspace(-2, 12, 15) - 0.1j
    g1 = ground.excitation_green(Hm, b, z)
    g2 = ground.lehmann_green(Hm, b, z)
    assert np.max(np.abs(g1 - g2)) < 1e-11
    zl = np.array([1e4 + 0.0j, -2e4 + 1.0j])
    gl = ground.excitation_green(Hm, b, zl)
    approx = (b @ b) / zl + (b @ (Hm @ b)) / zl ** 2
    assert np.max(np.abs(gl - approx) / np.abs(approx)) < 1e-6


def test_fermion_op_at_equals_whole_vector():
    """Entry-wise evaluation equals the whole-vector operator (L = 5, all
    sites, spins, c and c+)."""
    L, nu, nd = 5, 2, 3
    psi = inputs.random_unit_real(10 * 10, 12)
    for site, spin, create in itertools.product(range(L), range(2), (False, True)):
        full = ground.fermion_op(L, nu, nd, site, spin, create, psi)
        got = ground.fermion_op_at(L, nu, nd, site, spin, create, psi, np.arange(full.size))
        assert np.array_equal(got, full), (site, spin, create)


@pytest.mark.parametrize("L,nu,nd,periodic", [(5, 2, 3, True), (6, 3, 2, False), (4, 2, 2, True)])
def test_hubbard_rows_apply_equals_matrix(oracle_mod, L, nu, nd, periodic):
    """Row-wise H psi from the operators equals the C oracle's sector matrix."""
    H = hubbard(oracle_mod, L, nu, nd, t=0.7, U=3.0, V=1.3, periodic=periodic)
    psi = inputs.random_unit_real(H.shape[0], 13)
    rows = np.arange(H.shape[0])
    got = ground.hubbard_rows_apply(L, nu, nd, 0.7, 3.0, 1.3, periodic, psi, rows)
    assert np.allclose(got, H @ psi, rtol=0, atol=1e-14)


# ------------------------------------------------------------ Krylov subspace diagonalisation
def test_krylov_sd_chain_is_truncated_chain():
    """From the end site of an open chain the Lanczos basis is e_0, e_1, ...
    (alpha = 0, beta = |t|), so K_nu gives exactly the Green's function of the
    chain of nu sites: G_00 = closed form of the nu-site chain."""
    h = inputs.chain_csr(400, t=-1.0)
    b = np.zeros(h.n); b[0] = 1.0
    z = np.linspace(-2.5, 2.5, 11) + 0.05j
    res = ground.krylov_sd(h.scipy(), b, 30, z, b[None, :])
    assert res.nu == 30
    assert np.max(np.abs(res.G[0] - dense.chain_g00_exact(30, -1.0, z))) < 1e-12


def test_krylov_sd_complete_space_equals_dense():
    """nu = 2 N on 108 rows: past N steps the basis has lost orthogonality,
    but T's spectral measure (converged eigenvalues with their ghost copies)
    reproduces the dense Green's function (unit and dense projections); at
    nu = N it is not there yet."""
    h = inputs.anderson_csr(3, seed=4)           # 108 rows
    b = inputs.random_unit_real(h.n, 21)
    C = np.stack([b, np.eye(h.n)[5], inputs.random_unit_real(h.n, 22)])
    z = np.linspace(-5, 5, 9) + 0.3j
    ref = dense.green_dense(h.dense(), z, b.astype(np.complex128), C.astype(np.complex128))
    res = ground.krylov_sd(h.scipy(), b, 2 * h.n, z, C)
    assert np.max(np.abs(res.G - ref)) / np.max(np.abs(ref)) < 1e-10
    res = ground.krylov_sd(h.scipy(), b, 60, z, C)
    assert np.max(np.abs(res.G - ref)) / np.max(np.abs(ref)) > 1e-4


def test_krylov_sd_moments():
    """Gauss quadrature: with c = b the weights reproduce the moments
    b^T H^k b for k < 2 nu (nu = 6, before any loss of orthogonality)."""
    h = inputs.anderson_csr(4, seed=6)
    H = h.scipy()
    b = inputs.random_unit_real(h.n, 23)
    res = ground.krylov_sd(H, b, 6, [0.0 + 1j], b[None, :])
    v = b.copy()
    for k in range(12):
        mk = float(b @ v)
        assert abs(np.sum(res.weight[0] * res.ritz ** k) - mk) < 1e-9 * max(1.0, abs(mk)), k
        v = H @ v
