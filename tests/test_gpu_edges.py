"""Edge and degenerate cases through the C ABI: H = 0 and diagonal H (closed
forms), one row, the largest projection count, duplicate shifts, a real shift
outside the spectrum, and the size limits."""
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


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def relerr(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def solve(S, rowptr, col, val, shifts, b, tol, prec=0, **kw):
    h = S.scocg_create_csr(np.asarray(rowptr, np.int64), np.asarray(col, np.int32), np.asarray(val, np.float64),
                           opts=S.SolveOptions(precision=prec))
    try:
        G, info = S.scocg_solve(h, shifts, cuda(b), tol=tol, **kw)
        return G.cpu().numpy()[0], info
    finally:
        S.scocg_destroy(h)


@pytest.mark.parametrize("prec,bound", [(0, 1e-14), (2, 1e-13), (1, 1e-6)])
def test_zero_matrix_closed_form(S, prec, bound):
    """H = 0 (no stored entry): G_k = c^T b / z_k; the first step reaches r = 0."""
    n = 37
    b = inputs.random_unit_complex(n, 1)
    z = np.array([0.3 + 0.2j, -1.0 + 0.05j, 2.0 + 1.0j])
    g, info = solve(S, np.zeros(n + 1), [], [], z, b, 1e-12, prec, proj_vec=cuda(np.conj(b)[None, :]))
    assert info["status"] == 0
    assert relerr(g[0], (np.conj(b) @ b) / z) < bound


def test_diagonal_matrix_closed_form(S):
    """Diagonal H: G_k = sum_i c_i b_i / (z_k - h_i) (distinct h_i)."""
    n = 60
    rng = np.random.default_rng(3)
    hdiag = np.round(rng.uniform(-2, 2, n), 6)
    b = inputs.random_unit_complex(n, 2)
    c = rng.normal(size=n)
    z = np.linspace(-2.5, 2.5, 9) + 0.1j
    rp = np.arange(n + 1)
    g, info = solve(S, rp, np.arange(n), hdiag, z, b, 1e-13, 0, proj_vec=cuda(c[None, :].astype(np.complex128)))
    assert info["status"] == 0
    want = np.array([np.sum(c * b / (zk - hdiag)) for zk in z])
    assert relerr(g[0], want) < 1e-10


def test_single_row(S):
    """n = 1: G_k = c b / (z_k - h)."""
    z = np.array([0.5 + 0.1j, 3.0 + 0.01j])
    g, info = solve(S, [0, 1], [0], [0.7], z, np.array([2.0 + 1.0j]), 1e-13, 0, proj_idx=[0])
    assert info["status"] == 0
    assert relerr(g[0], (2.0 + 1.0j) / (z - 0.7)) < 1e-14


def test_max_projections_and_duplicate_shifts(S, oracle_mod):
    """32 dense projections (the limit) after 8 iterations (before the extreme Ritz
    values of these 256 rows converge) against the
    oracle; a repeated shift gives bit-identical columns."""
    h = inputs.anderson_csr(4, seed=41)
    b = inputs.random_unit_complex(h.n, 3)
    C = np.stack([inputs.random_unit_complex(h.n, 100 + m) for m in range(32)])
    z = np.array([0.3 + 0.1j, -1.2 + 0.1j, 0.3 + 0.1j, 2.0 + 0.1j])
    hh = S.scocg_create_csr(h.rowptr, h.col, h.val, opts=S.SolveOptions(max_iter=8, seed=0))
    try:
        G, info = S.scocg_solve(hh, z, cuda(b), proj_vec=cuda(C), tol=0.0)
        with pytest.raises(S.ScocgError):
            S.scocg_solve(hh, z, cuda(b), proj_vec=cuda(np.concatenate([C, C[:1]])), tol=0.0)
        with pytest.raises(S.ScocgError):
            S.scocg_solve(hh, np.linspace(-1, 1, 4097) + 0.1j, cuda(b), proj_idx=[0], tol=0.0)
    finally:
        S.scocg_destroy(hh)
    G = G.cpu().numpy()[0]
    ref = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, z, b, proj_vec=list(C), tol=0.0, max_iter=8, seed=0)
    # per shift, relative to the largest |G| over the 32 projections: random
    # dense projections put some G_mk near zero
    err = np.max(np.abs(G - ref.G), axis=0) / np.max(np.abs(ref.G), axis=0)
    assert err.max() < 1e-10
    assert np.array_equal(G[:, 0], G[:, 2])


def test_real_shift_outside_spectrum(S, oracle_mod):
    """Im z = 0 above the spectrum (z - H positive definite): converges like CG."""
    h = inputs.anderson_csr(3, seed=43)
    lo, hi = inputs.spectral_bounds(h)
    b = inputs.random_unit_complex(h.n, 4)
    z = np.array([hi + 1.0, hi + 3.0, lo - 2.0])
    g, info = solve(S, h.rowptr, h.col, h.val, z, b, 1e-13, 0, proj_vec=cuda(np.conj(b)[None, :]))
    assert info["status"] == 0
    ref = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, z, b, proj_vec=[np.conj(b)], tol=1e-13)
    assert relerr(g[0], ref.G[0]) < 1e-11
