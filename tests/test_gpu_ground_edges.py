"""Edge cases of the ground-state, excitation and Krylov-subspace entry points,
each against a closed form: a 1-row matrix, one Krylov step, a start vector
that already spans an invariant subspace, and excitations into and out of the
empty and the completely filled sectors."""
import numpy as np
import pytest

from paper_0802_0748_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0802_0748_gb300 import scocg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return scocg


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def one_row(S, a):
    return S.scocg_create_csr(np.array([0, 1]), np.array([0], dtype=np.int32), np.array([a]))


def test_ground_state_one_row(S):
    """H = [2.5]: E = 2.5, psi = +-1, residual 0, one Lanczos step per cycle."""
    h = one_row(S, 2.5)
    try:
        e0, psi, info = S.scocg_ground_state(h, dev([-3.0]), m=4, tol=1e-14)
    finally:
        S.scocg_destroy(h)
    assert info["status"] == 0 and e0 == 2.5 and abs(abs(psi.item()) - 1.0) < 1e-15
    assert info["lanczos_steps"] == 1


def test_krylov_one_step_closed_form(S):
    """nu = 1: T = [v0^T H v0], weight = c^T b, G(z) = c^T b / (z - b^T H b / b^T b)."""
    h_csr = inputs.anderson_csr(4, seed=2)
    b = inputs.random_unit_real(h_csr.n, 3) * 2.0
    z = np.array([0.3 + 0.2j, -4.0 + 1.0j, 7.0 + 0.01j])
    a0 = float(b @ (h_csr.scipy() @ b) / (b @ b))
    h = S.scocg_create_csr(h_csr.rowptr, h_csr.col, h_csr.val)
    try:
        G, r, w, info = S.scocg_krylov_sd(h, dev(b), 1, z, proj_idx=[7, 100])
    finally:
        S.scocg_destroy(h)
    assert info["nu_used"] == 1
    assert abs(r.item() - a0) < 1e-13 * max(1.0, abs(a0))
    ref = np.stack([b[7] / (z - a0), b[100] / (z - a0)])
    assert np.max(np.abs(G.cpu().numpy() - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("layout", [0, 1])
def test_krylov_invariant_start(S, layout):
    """b = an eigenvector of H: the recursion stops after one step (beta_0
    vanishes), one Ritz value = its eigenvalue, G = c^T b / (z - e).  Both the
    one-launch recursion (layout 0) and one launch per operation (layout 1)."""
    h_csr = inputs.anderson_csr(3, seed=8)
    E, U = np.linalg.eigh(h_csr.dense())
    b = U[:, 5]
    z = np.linspace(-3, 3, 7) + 0.1j
    h = S.scocg_create_csr(h_csr.rowptr, h_csr.col, h_csr.val, opts=S.SolveOptions(layout=layout))
    try:
        G, r, w, info = S.scocg_krylov_sd(h, dev(b), 40, z, proj_idx=[11])
    finally:
        S.scocg_destroy(h)
    assert info["nu_used"] == 1
    assert abs(r.item() - E[5]) < 1e-12
    assert np.max(np.abs(G.cpu().numpy()[0] - b[11] / (z - E[5]))) < 1e-12 * np.max(np.abs(b[11] / (z - E[5])))


def test_excite_to_empty_and_full_sectors(S):
    """L = 5: c_{i up} from the one-up-electron sector to the empty up sector,
    and c+_{i dn} from four down electrons to the full down sector, against
    the oracle's Jordan-Wigner operator, bit for bit."""
    from oracle import ground
    L = 5
    cases = [((1, 2), (0, 2), 0, False), ((2, 4), (2, 5), 1, True)]
    for (nu, nd), (tu, td), spin, create in cases:
        src = S.scocg_create_hubbard(L, nu, nd, 1.0, 4.0, 1.0, True)
        dst = S.scocg_create_hubbard(L, tu, td, 1.0, 4.0, 1.0, True)
        try:
            import math
            n = math.comb(L, nu) * math.comb(L, nd)
            psi = inputs.random_unit_real(n, 50 + spin)
            for site in range(L):
                out = S.scocg_excite(src, dst, site, spin, create, dev(psi)).cpu().numpy()
                ref = ground.fermion_op(L, nu, nd, site, spin, create, psi)
                assert np.array_equal(out.real, ref), (site, spin, create)
        finally:
            S.scocg_destroy(src)
            S.scocg_destroy(dst)
