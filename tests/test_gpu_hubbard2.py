"""Two-orbital extended Hubbard model of Sec. IV.B (scocg_create_hubbard2)
through the C ABI against the oracle's literal Jordan-Wigner construction.

With the synthetic sqrt(8) x sqrt(8) values every matrix element is a dyadic
rational, so H x for a small-integer x is exact in any summation order: the
applies are compared bit for bit (FP64, complex64 and compensated), including
sampled rows of the paper's 6 up / 6 down sector (64,128,064 states) computed
one by one by the oracle.  Generic (non-dyadic) hoppings on a two-site cluster
check every term at the FP64 rounding level; solves are compared with the
oracle's shifted COCG on the oracle's CSR (fixed iterations before Ritz
convergence, and converged), and the ground state with ARPACK."""
import math

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
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def csr_product(oracle_mod, model, nu, nd, x):
    import scipy.sparse as sp
    rp, c, v = oracle_mod.hubbard2_csr(model, nu, nd)
    n = rp.size - 1
    return sp.csr_matrix((v, c, rp), shape=(n, n)) @ x, (rp, c, v)


def int_vector(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(-8, 9, n) + 1j * rng.integers(-8, 9, n)).astype(np.complex128)


def to_df(x):
    return np.stack([x.real, x.imag, np.zeros(x.size), np.zeros(x.size)], axis=1).astype(np.float32)


def from_df(v):
    v = v.astype(np.float64)
    return (v[:, 0] + v[:, 2]) + 1j * (v[:, 1] + v[:, 3])


@pytest.mark.parametrize("nu,nd", [(2, 2), (3, 1), (1, 0)])
def test_apply_bit_exact_sqrt8(S, oracle_mod, nu, nd):
    """y = (z - H) x on the sqrt(8) x sqrt(8) cluster, integer x: bit-exact in
    FP64, complex64 and compensated FP32 against the oracle's CSR product."""
    m = inputs.eg_model()
    h = S.scocg_create_hubbard2(m, nu, nd)
    try:
        n = S.scocg_dim(h)
        assert n == math.comb(16, nu) * math.comb(16, nd)
        x = int_vector(n, 3)
        ref, _ = csr_product(oracle_mod, m, nu, nd, x)
        z = 0.5 + 0.25j
        want = z * x - ref
        y = S.scocg_apply(h, z, cuda(x)).cpu().numpy()
        assert np.array_equal(y, want)
        y32 = S.scocg_apply(h, z, cuda(x.astype(np.complex64)), precision=S.MIXED).cpu().numpy()
        assert np.array_equal(y32.astype(np.complex128), want)
        ydf = from_df(S.scocg_apply(h, z, cuda(to_df(x)), precision=S.MIXED_DF).cpu().numpy())
        assert np.array_equal(ydf, want)
    finally:
        S.scocg_destroy(h)


@pytest.mark.parametrize("nu,nd", [(1, 1), (2, 1), (2, 2), (3, 1), (1, 3)])
def test_apply_generic_two_site(S, oracle_mod, nu, nd):
    """Two sites with generic hoppings and interaction values: every term at
    the FP64 rounding level."""
    m = inputs.eg_model(bonds=[(0, 1)], dirs=[0], U=3.1, Up=1.7, J=0.6, Jp=0.45, V=0.8)
    m["bond_t"] = np.random.default_rng(3).normal(size=(1, 2, 2)).tolist()
    h = S.scocg_create_hubbard2(m, nu, nd)
    try:
        n = S.scocg_dim(h)
        x = inputs.random_unit_complex(n, 5)
        ref, _ = csr_product(oracle_mod, m, nu, nd, x)
        y = S.scocg_apply(h, 0.0, cuda(x)).cpu().numpy()
        assert np.max(np.abs(y + ref)) <= 1e-14 * np.max(np.abs(ref))
    finally:
        S.scocg_destroy(h)


def test_full_sector_sampled_rows_bit_exact(S, oracle_mod):
    """The paper's sector (sqrt(8) x sqrt(8), 6 up 6 down, (16 C 6)^2 =
    64,128,064 states): 4,000 sampled rows of H x (integer x) bit-exact
    against the oracle's row-by-row construction, FP64 and compensated."""
    m = inputs.eg_model()
    h = S.scocg_create_hubbard2(m, 6, 6)
    try:
        n = S.scocg_dim(h)
        assert n == 64128064
        x = int_vector(n, 11)
        rows = np.unique(np.concatenate([np.random.default_rng(12).choice(n, 4000, replace=False),
                                         [0, 1, n // 2, n - 2, n - 1]]))
        ref = oracle_mod.hubbard2_rows(m, 6, 6, rows, x)
        xd = cuda(x)
        y = S.scocg_apply(h, 0.0, xd)
        assert np.array_equal(y.cpu().numpy()[rows], -ref)
        del y
        xf = cuda(to_df(x))
        del xd
        ydf = S.scocg_apply(h, 0.0, xf, precision=S.MIXED_DF).cpu().numpy()
        assert np.array_equal(from_df(ydf[rows]), -ref)
    finally:
        S.scocg_destroy(h)
        torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", [0, 2])
def test_fixed_iterations_match_oracle(S, oracle_mod, prec):
    """3 up 3 down on the sqrt(8) x sqrt(8) cluster (313,600 states), 16 shifts,
    25 iterations (before any Ritz value converges): G element by element
    against the oracle's shifted COCG on its CSR.  The bound is set by the
    problem's own sensitivity to rounding: on the oracle itself a 2^-53
    relative perturbation of b moves this G by up to 1.2e-10 after 12
    iterations and 5.2e-10 after 25 (three draws), so FP64 and compensated
    results, whose sums run in another order, are held to 2e-9."""
    bound = 2e-9
    m = inputs.eg_model()
    wl = inputs.workload("hubbard2", "medium")
    rp, c, v = oracle_mod.hubbard2_csr(m, 3, 3)
    shifts = wl.shifts[::8]
    b = wl.rhs[0]
    n_it = 25
    h = S.scocg_create_hubbard2(m, 3, 3, opts=S.SolveOptions(precision=prec, max_iter=n_it))
    try:
        G, info = S.scocg_solve(h, shifts, cuda(b), proj_vec=cuda(wl.proj_vec), tol=0.0)
    finally:
        S.scocg_destroy(h)
    seed = oracle_mod.default_seed(shifts)
    ref = oracle_mod.shifted_cocg(rp, c, v, shifts, b, proj_vec=wl.proj_vec, tol=0.0, max_iter=n_it, seed=seed)
    assert info["iters"] == n_it
    assert relerr(G.cpu().numpy()[0], ref.G) < bound


def test_converged_small_sector_and_ground_state(S, oracle_mod):
    """2 up 2 down (14,400 states): converged G (FP64, residual 1e-12) against
    the oracle's converged solve, and the ground-state energy against ARPACK
    on the oracle's CSR."""
    m = inputs.eg_model()
    wl = inputs.workload("hubbard2", "small")
    rp, c, v = oracle_mod.hubbard2_csr(m, 2, 2)
    shifts = wl.shifts[::4]
    b = wl.rhs[0]
    h = S.scocg_create_hubbard2(m, 2, 2)
    try:
        G, info = S.scocg_solve(h, shifts, cuda(b), proj_vec=cuda(wl.proj_vec), tol=1e-12)
        v0 = cuda(inputs.random_unit_real(rp.size - 1, 4))
        E, psi, ginfo = S.scocg_ground_state(h, v0, m=60, cg_steps=30, tol=1e-9)
    finally:
        S.scocg_destroy(h)
    ref = oracle_mod.shifted_cocg(rp, c, v, shifts, b, proj_vec=wl.proj_vec, tol=1e-12)
    assert info["status"] == 0
    assert relerr(G.cpu().numpy()[0], ref.G) < 1e-10
    import scipy.sparse as sp
    from scipy.sparse.linalg import eigsh
    n = rp.size - 1
    e0 = eigsh(sp.csr_matrix((v, c, rp), shape=(n, n)), k=1, which="SA", tol=1e-13)[0][0]
    assert ginfo["status"] == 0 and abs(E - e0) < 1e-10 * max(1.0, abs(e0))


def test_invalid_models(S):
    m = inputs.eg_model()
    for bad in (dict(m, bonds=[(0, 0)] + m["bonds"][1:]),
                dict(m, bonds=[(0, 9)] + m["bonds"][1:]),
                dict(m, U=float("nan"))):
        with pytest.raises(S.ScocgError) as e:
            S.scocg_create_hubbard2(bad, 2, 2)
        assert e.value.code == S.ERR_INVALID
    # a site in eight bonds exceeds the 4-bit neighbour sums
    star = {"n_sites": 9, "bonds": [(0, j) for j in range(1, 9)], "bond_t": np.ones((8, 2, 2)).tolist(),
            "U": 1.0, "Up": 1.0, "J": 0.0, "Jp": 0.0, "V": 1.0}
    with pytest.raises(S.ScocgError):
        S.scocg_create_hubbard2(star, 1, 1)
    with pytest.raises(S.ScocgError):
        S.scocg_create_hubbard2(m, 17, 0)
