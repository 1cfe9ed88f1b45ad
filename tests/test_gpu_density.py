"""Density-matrix elements by the Fermi integral of Eq. densityM through the C
ABI: the GPU quadrature equals the oracle's quadrature of its own Green's
functions on the same grid (FP64, 1e-10), and approaches the exact eigenstate
sum within the broadening error."""
import numpy as np
import pytest

from paper_0802_0748_gb300 import inputs
from oracle import dense

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


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def grid(emin, emax, n):
    return np.linspace(emin, emax, n)


def test_density_matches_oracle_quadrature_fp64(S, oracle_mod):
    """Anderson 4^3 x 4 (256 rows), local densities rho_jj at three sites (block
    mode, unit right-hand sides), mu = 0.2, kT = 0.1, delta = 0.05, 512 points."""
    h = inputs.anderson_csr(4, seed=21)
    lo, hi = inputs.spectral_bounds(h)
    emin, emax, nq, delta, mu, kT = lo - 1.0, hi + 1.0, 512, 0.05, 0.2, 0.1
    sites = np.array([0, 77, 200])
    rhs = np.zeros((3, h.n), dtype=np.complex128)
    rhs[np.arange(3), sites] = 1.0
    hh = S.scocg_create_csr(h.rowptr, h.col, h.val)
    try:
        rho, info = S.scocg_density(hh, mu, kT, delta, emin, emax, nq, cuda(rhs), proj_idx=sites[:, None],
                                    tol=1e-13)
    finally:
        S.scocg_destroy(hh)
    assert info["status"] == 0
    rho = rho.cpu().numpy()[:, 0]
    e = grid(emin, emax, nq)
    for j, s in enumerate(sites):
        ref = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, e + 1j * delta, rhs[j], proj_idx=[int(s)], tol=1e-13)
        want = dense.density_quadrature(ref.G[0], e, mu, kT)
        assert abs(rho[j] - want) <= 1e-10 * abs(want), j


def test_density_dense_projection_and_exact_limit(S):
    """Chain of 64 sites at mu = 0 (half filling of a bipartite lattice): every
    site holds 1/2; with c = conj(b) for a random b the quadrature approaches
    b^H rho b of the eigenstate sum as the grid and broadening are refined."""
    L = 64
    h = inputs.chain_csr(L)
    b = inputs.random_unit_complex(L, 3)
    H = h.dense()
    exact = dense.density_exact(H, b, [np.conj(b)], 0.0, 0.05)[0]
    e0 = np.eye(L, dtype=np.complex128)[10]
    hh = S.scocg_create_csr(h.rowptr, h.col, h.val)
    try:
        errs = []
        for delta in (0.04, 0.02):
            nq = int(round(10.0 / (delta / 8))) + 1
            nq = min(nq, 4096)
            rho, info = S.scocg_density(hh, 0.0, 0.05, delta, -5.0, 5.0, nq, cuda(b),
                                        proj_vec=cuda(np.conj(b)[None, :]), tol=1e-12)
            assert info["status"] == 0
            errs.append(abs(rho.cpu().numpy()[0, 0] - exact))
        r_site, _ = S.scocg_density(hh, 0.0, 0.05, 0.02, -5.0, 5.0, 4001, cuda(e0), proj_idx=[10], tol=1e-12)
    finally:
        S.scocg_destroy(hh)
    assert errs[1] < 0.7 * errs[0] and errs[1] < 2e-2
    # half filling: 1/2 less the Lorentzian tails outside the window (~ delta / (pi * 3))
    assert abs(r_site.cpu().numpy()[0, 0] - 0.5) < 5e-3


def test_density_invalid(S):
    h = inputs.chain_csr(8)
    hh = S.scocg_create_csr(h.rowptr, h.col, h.val)
    try:
        e0 = cuda(np.eye(8)[0].astype(np.complex128))
        for args in ((0.0, 0.1, 0.0, -3.0, 3.0, 64), (0.0, 0.1, 0.05, 3.0, -3.0, 64), (0.0, -1.0, 0.05, -3.0, 3.0, 64),
                     (0.0, 0.1, 0.05, -3.0, 3.0, 1)):
            with pytest.raises(RuntimeError):
                S.scocg_density(hh, *args, e0, proj_idx=[0])
    finally:
        S.scocg_destroy(hh)
