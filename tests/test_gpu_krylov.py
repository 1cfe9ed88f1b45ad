"""Green's functions by subspace diagonalisation in the Krylov subspace
(Sec. III.B) through the C ABI, against the oracle.

Without reorthogonalization the Lanczos recursion is forward unstable once a
Ritz value converges: two correct implementations with different rounding
then place the ghost copies of converged eigenvalues differently.  A
rounding-level change of b moves G by ~1e-14 up to 40 steps on the 4^3 x 4
matrix and by 1e-3 at 100 steps, so element-wise parity with the oracle is
tested at nu <= 40 and larger nu through what holds for any correct
recursion: the truncated-chain closed form, the dense G once the spectral
measure of T has converged, the moments b^T H^k b, and sum rules.
"""
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


def csr_handle(S, h):
    return S.scocg_create_csr(h.rowptr, h.col, h.val)


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_chain_closed_form(S):
    """Open chain of 4,096 sites from its end site: the Lanczos basis is
    e_0, e_1, ... exactly, so K_nu gives the nu-site chain's G_00 (closed form)."""
    from oracle import dense
    h_csr = inputs.chain_csr(4096, t=-1.0)
    b = np.zeros(h_csr.n); b[0] = 1.0
    z = np.linspace(-2.5, 2.5, 33) + 0.05j
    h = csr_handle(S, h_csr)
    try:
        G, ritz, w, info = S.scocg_krylov_sd(h, dev(b), 50, z, proj_idx=[0])
    finally:
        S.scocg_destroy(h)
    assert info["nu_used"] == 50
    assert np.max(np.abs(G.cpu().numpy()[0] - dense.chain_g00_exact(50, -1.0, z))) < 1e-12
    # the Ritz values of the 50-site chain: 2 cos(pi a / 51)
    ref = np.sort(-2.0 * np.cos(np.pi * np.arange(1, 51) / 51))
    assert np.max(np.abs(ritz.cpu().numpy() - ref)) < 1e-13


@pytest.mark.parametrize("nu", [12, 40])
def test_matches_oracle_before_orthogonality_is_lost(S, nu):
    """4^3 x 4 Anderson matrix (256 rows), random real b, unit and dense
    projections: G, Ritz values and weights equal the oracle's."""
    from oracle import ground
    h_csr = inputs.anderson_csr(4, seed=5)
    b = inputs.random_unit_real(h_csr.n, 30)
    C = np.stack([b, np.eye(h_csr.n)[3], inputs.random_unit_real(h_csr.n, 31)])
    z = np.linspace(-7, 7, 15) + 0.1j
    ref = ground.krylov_sd(h_csr.scipy(), b, nu, z, C)
    h = csr_handle(S, h_csr)
    try:
        Gd, rd, wd, idn = S.scocg_krylov_sd(h, dev(b), nu, z, proj_vec=dev(C))
        Gu, ru, wu, iun = S.scocg_krylov_sd(h, dev(b), nu, z, proj_idx=[3])
    finally:
        S.scocg_destroy(h)
    assert idn["nu_used"] == nu and iun["nu_used"] == nu
    scale = np.max(np.abs(ref.ritz))
    assert np.max(np.abs(rd.cpu().numpy() - ref.ritz)) < 1e-12 * scale
    assert np.max(np.abs(Gd.cpu().numpy() - ref.G)) / np.max(np.abs(ref.G)) < 1e-10
    assert np.max(np.abs(wd.cpu().numpy() - ref.weight)) < 1e-10 * np.max(np.abs(ref.weight))
    assert np.max(np.abs(Gu.cpu().numpy()[0] - ref.G[1])) / np.max(np.abs(ref.G[1])) < 1e-10


def test_converged_measure_equals_dense(S):
    """108 rows, nu = 2 N (past N steps the ghosts carry the weight): G equals
    the dense Green's function; with c = b the weights sum to ||b||^2."""
    from oracle import dense
    h_csr = inputs.anderson_csr(3, seed=4)
    b = inputs.random_unit_real(h_csr.n, 21) * 3.0
    C = np.stack([b, np.eye(h_csr.n)[5]])
    z = np.linspace(-5, 5, 9) + 0.3j
    h = csr_handle(S, h_csr)
    try:
        G, ritz, w, info = S.scocg_krylov_sd(h, dev(b), 2 * h_csr.n, z, proj_vec=dev(C))
    finally:
        S.scocg_destroy(h)
    ref = dense.green_dense(h_csr.dense(), z, b.astype(np.complex128), C.astype(np.complex128))
    assert np.max(np.abs(G.cpu().numpy() - ref)) / np.max(np.abs(ref)) < 1e-9
    assert abs(w.cpu().numpy()[0].sum() - b @ b) < 1e-11 * (b @ b)


def test_hubbard_handle_matches_oracle(S, oracle_mod):
    """Matrix-free Hubbard ring L=8, 3 up 3 down (3,136 states), nu = 30,
    against the oracle on the sector matrix built from the Fock-space
    definition."""
    import scipy.sparse as sp
    from oracle import ground
    rowptr, col, val = oracle_mod.hubbard_csr(8, 3, 3, 1.0, 4.0, 1.0, True)
    n = rowptr.size - 1
    H = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    b = inputs.random_unit_real(n, 33)
    z = np.linspace(-6, 16, 12) + 0.2j
    ref = ground.krylov_sd(H, b, 30, z, np.stack([b, np.eye(n)[17]]))
    h = S.scocg_create_hubbard(8, 3, 3, 1.0, 4.0, 1.0, True)
    try:
        G, ritz, w, info = S.scocg_krylov_sd(h, dev(b), 30, z, proj_idx=[17])
        G2, _, _, _ = S.scocg_krylov_sd(h, dev(b), 30, z, proj_vec=dev(b[None, :]))
    finally:
        S.scocg_destroy(h)
    assert np.max(np.abs(G.cpu().numpy()[0] - ref.G[1])) / np.max(np.abs(ref.G[1])) < 1e-10
    assert np.max(np.abs(G2.cpu().numpy()[0] - ref.G[0])) / np.max(np.abs(ref.G[0])) < 1e-10


def test_moments_at_batch_size(S):
    """The 32^3 x 4 matrix (131,072 rows), nu = 200 from unit vectors e_j: the
    weights reproduce b^T H^k b for k <= 9 (scipy matvecs), and sum to 1."""
    h_csr = inputs.anderson_csr(32, seed=1)
    H = h_csr.scipy()
    h = csr_handle(S, h_csr)
    try:
        for j in (0, 77_777):
            b = np.zeros(h_csr.n); b[j] = 1.0
            G, ritz, w, info = S.scocg_krylov_sd(h, dev(b), 200, [0.1j], proj_idx=[j])
            e = ritz.cpu().numpy(); wt = w.cpu().numpy()[0]
            assert info["nu_used"] == 200
            v = b.copy()
            for k in range(10):
                mk = float(b @ v)
                scale = float(np.linalg.norm(v))
                assert abs(np.sum(wt * e ** k) - mk) < 1e-11 * max(1.0, scale), (j, k)
                v = H @ v
    finally:
        S.scocg_destroy(h)


def test_one_launch_recursion_equals_launch_per_step(S):
    """Unit projections on the 4x4-blocked layout run the whole recursion in
    one cooperative launch; forcing the plain CSR layout runs one launch per
    operation.  Same G, Ritz values and weights (nu = 30, before orthogonality
    is lost), on the 8^3 x 4 matrix (2,048 rows, several CTAs)."""
    h_csr = inputs.anderson_csr(8, seed=9)
    b = inputs.random_unit_real(h_csr.n, 40)
    z = np.linspace(-7, 7, 21) + 0.05j
    out = []
    for layout in (0, 1):
        h = S.scocg_create_csr(h_csr.rowptr, h_csr.col, h_csr.val, opts=S.SolveOptions(layout=layout))
        try:
            G, r, w, info = S.scocg_krylov_sd(h, dev(b), 30, z, proj_idx=[1, 700])
        finally:
            S.scocg_destroy(h)
        assert info["nu_used"] == 30
        out.append((G.cpu().numpy(), r.cpu().numpy(), w.cpu().numpy()))
    (G0, r0, w0), (G1, r1, w1) = out
    assert np.max(np.abs(r0 - r1)) < 1e-12 * np.max(np.abs(r1))
    assert np.max(np.abs(G0 - G1)) < 1e-10 * np.max(np.abs(G1))
    assert np.max(np.abs(w0 - w1)) < 1e-10 * np.max(np.abs(w1))


def test_invalid_arguments(S):
    h_csr = inputs.anderson_csr(3, seed=4)
    h = csr_handle(S, h_csr)
    b = dev(inputs.random_unit_real(h_csr.n, 1))
    try:
        for kw in ({"nu": 0}, {"nu": 2000}):
            with pytest.raises(S.ScocgError):
                S.scocg_krylov_sd(h, b, kw["nu"], [0.1j], proj_idx=[0])
        with pytest.raises(S.ScocgError):
            S.scocg_krylov_sd(h, b, 10, [0.1j], proj_idx=[h_csr.n])
        with pytest.raises(S.ScocgError):
            S.scocg_krylov_sd(h, torch.zeros_like(b), 10, [0.1j], proj_idx=[0])
    finally:
        S.scocg_destroy(h)


def krsd_single(S, h, B, nu, z, pidx):
    out, used = [], []
    for r in range(B.shape[0]):
        G, ritz, w, info = S.scocg_krylov_sd(h, dev(B[r]), nu, z, proj_idx=pidx[r])
        out.append(G.cpu().numpy())
        used.append(info["nu_used"])
    return np.stack(out), np.asarray(used)


@pytest.mark.parametrize("nrhs", [5, 12, 19, 40])
def test_multi_equals_single_and_oracle(S, nrhs):
    """Several right-hand sides in one launch (T = 8, 16, 32 slots; 40 = a
    full tile and a ragged one) on the 8^3 x 4 matrix, nu = 30 (before
    orthogonality is lost): every right-hand side's G equals the
    one-right-hand-side recursion's and, for three of them, the oracle's."""
    from oracle import ground
    h_csr = inputs.anderson_csr(8, seed=9)
    n = h_csr.n
    rng = np.random.default_rng(nrhs)
    sites = rng.choice(n, nrhs, replace=False)
    B = np.zeros((nrhs, n))
    B[np.arange(nrhs), sites] = 1.0
    B[::3] = np.stack([inputs.random_unit_real(n, 100 + r) for r in range(0, nrhs, 3)])
    pidx = np.stack([sites, rng.choice(n, nrhs)], axis=1)
    z = np.linspace(-7, 7, 21) + 0.05j
    h = csr_handle(S, h_csr)
    try:
        Gm, used, info = S.scocg_krylov_sd_multi(h, dev(B), 30, z, pidx)
        Gs, used_s = krsd_single(S, h, B, 30, z, pidx)
    finally:
        S.scocg_destroy(h)
    Gm = Gm.cpu().numpy()
    assert np.array_equal(used, used_s) and np.all(used == 30)
    for r in range(nrhs):
        assert np.max(np.abs(Gm[r] - Gs[r])) < 1e-10 * np.max(np.abs(Gs[r])), r
    for r in (0, 1, nrhs - 1):
        C = np.eye(n)[pidx[r]]
        ref = ground.krylov_sd(h_csr.scipy(), B[r], 30, z, C)
        assert np.max(np.abs(Gm[r] - ref.G)) < 1e-10 * np.max(np.abs(ref.G)), r


def test_multi_slots_end_on_their_own(S):
    """H the direct sum of a 3^3 x 4 matrix, a 4^3 x 4 matrix and one
    isolated 4 x 4 block (108 + 256 + 4 rows): a right-hand side inside the
    4 x 4 block spans 4 Krylov vectors, so its slot ends (beta vanishes)
    after at most 4 steps while the others run on (nu = 600); every
    right-hand side's G then equals its dense Green's function, with FP64
    and with compensated arithmetic."""
    import scipy.sparse as sp
    from oracle import dense
    a, b_ = inputs.anderson_csr(3, seed=4), inputs.anderson_csr(4, seed=6)
    small = np.array([[0.5, 0.25, 0.0, -0.125], [0.25, -1.0, 0.375, 0.0],
                      [0.0, 0.375, 1.5, 0.25], [-0.125, 0.0, 0.25, -0.5]])
    Hs = sp.block_diag([a.scipy(), b_.scipy(), sp.csr_matrix(small)], format="csr")
    Hs.sort_indices()
    n = Hs.shape[0]
    B = np.zeros((6, n))
    B[0, 5] = B[1, 150] = 1.0
    B[2, :108] = inputs.random_unit_real(108, 7)
    B[3, 365] = 1.0
    B[4] = inputs.random_unit_real(n, 9)
    B[5, 364:] = [0.5, -0.5, 0.5, 0.5]
    pidx = np.array([[5, 7], [150, 151], [0, 100], [365, 366], [3, 250], [364, 367]])
    z = np.linspace(-6, 6, 13) + 0.2j
    Hd = Hs.toarray()
    for prec, bound in ((0, 1e-9), (2, 1e-8)):
        h = S.scocg_create_csr(Hs.indptr.astype(np.int64), Hs.indices.astype(np.int64), Hs.data,
                               opts=S.SolveOptions(precision=prec))
        try:
            Gm, used, info = S.scocg_krylov_sd_multi(h, dev(B), 600, z, pidx)
        finally:
            S.scocg_destroy(h)
        Gm = Gm.cpu().numpy()
        assert used[3] <= 4 and used[5] <= 4
        assert all(used[r] > 100 for r in (0, 1, 2, 4))
        for r in range(6):
            ref = dense.green_dense(Hd, z, B[r].astype(np.complex128), np.eye(n)[pidx[r]].astype(np.complex128))
            assert np.max(np.abs(Gm[r] - ref)) < bound * np.max(np.abs(ref)), (prec, r)


def test_multi_on_other_layouts_and_refusals(S):
    """The plain CSR layout and a Hubbard handle run the one-right-hand-side
    recursion per right-hand side (same G as calling it); a zero right-hand
    side or an index out of range is refused."""
    h_csr = inputs.anderson_csr(4, seed=5)
    n = h_csr.n
    B = np.stack([inputs.random_unit_real(n, 50), np.eye(n)[9]])
    pidx = np.array([[1], [9]])
    z = np.linspace(-7, 7, 9) + 0.1j
    h = S.scocg_create_csr(h_csr.rowptr, h_csr.col, h_csr.val, opts=S.SolveOptions(layout=1))
    try:
        Gm, used, _ = S.scocg_krylov_sd_multi(h, dev(B), 25, z, pidx)
        Gs, used_s = krsd_single(S, h, B, 25, z, pidx)
        assert np.array_equal(Gm.cpu().numpy(), Gs) and np.array_equal(used, used_s)
        with pytest.raises(S.ScocgError):
            S.scocg_krylov_sd_multi(h, dev(np.zeros((1, n))), 10, z, [[0]])
        with pytest.raises(S.ScocgError):
            S.scocg_krylov_sd_multi(h, dev(B), 10, z, [[0], [n]])
    finally:
        S.scocg_destroy(h)
    h = csr_handle(S, h_csr)
    try:
        with pytest.raises(S.ScocgError):
            S.scocg_krylov_sd_multi(h, dev(np.stack([B[0], np.zeros(n)])), 10, z, pidx)
    finally:
        S.scocg_destroy(h)
    hb = S.scocg_create_hubbard(6, 2, 2, 1.0, 4.0, 1.0, True)
    try:
        nh = S.scocg_dim(hb)
        Bh = np.stack([inputs.random_unit_real(nh, 60), inputs.random_unit_real(nh, 61)])
        Gm, used, _ = S.scocg_krylov_sd_multi(hb, dev(Bh), 20, z, [[3], [4]])
        Gs, _ = krsd_single(S, hb, Bh, 20, z, [[3], [4]])
        assert np.array_equal(Gm.cpu().numpy(), Gs)
    finally:
        S.scocg_destroy(hb)


def test_multi_compensated_matches_fp64_and_oracle(S):
    """The compensated recursion (SCOCG_MIXED_DF handle: FP32 blocks of H,
    vectors as float pairs, FP64 step scalars) on the 8^3 x 4 matrix, 19
    right-hand sides, nu = 30: G within 1e-9 of the FP64 recursion's and of
    the oracle's (the values of H are FP32-exact)."""
    from oracle import ground
    h_csr = inputs.anderson_csr(8, seed=9)
    n = h_csr.n
    rng = np.random.default_rng(3)
    sites = rng.choice(n, 19, replace=False)
    B = np.stack([inputs.random_unit_real(n, 200 + r) for r in range(19)])
    B[1::2] = 0.0
    B[np.arange(1, 19, 2), sites[1::2]] = 1.0
    pidx = np.stack([sites, rng.choice(n, 19)], axis=1)
    z = np.linspace(-7, 7, 21) + 0.05j
    out = {}
    for prec in (0, 2):
        h = S.scocg_create_csr(h_csr.rowptr, h_csr.col, h_csr.val, opts=S.SolveOptions(precision=prec))
        try:
            G, used, _ = S.scocg_krylov_sd_multi(h, dev(B), 30, z, pidx)
        finally:
            S.scocg_destroy(h)
        assert np.all(used == 30)
        out[prec] = G.cpu().numpy()
    for r in range(19):
        assert np.max(np.abs(out[2][r] - out[0][r])) < 1e-9 * np.max(np.abs(out[0][r])), r
    for r in (0, 1, 18):
        ref = ground.krylov_sd(h_csr.scipy(), B[r], 30, z, np.eye(n)[pidx[r]])
        assert np.max(np.abs(out[2][r] - ref.G)) < 1e-9 * np.max(np.abs(ref.G)), r


@pytest.mark.parametrize("prec", [0, 2])
def test_multi_one_step_closed_form(S, prec):
    """nu = 1 from b = e_j with projection e_j: T = [H_jj], so G = 1 / (z -
    H_jj) exactly, for a single right-hand side (one slot of eight used) and
    for 33 of them (a full tile of 32 and a tile with one)."""
    h_csr = inputs.anderson_csr(6, seed=3)
    n = h_csr.n
    Hd = h_csr.dense()
    z = np.linspace(-3, 3, 7) + 0.25j
    h = S.scocg_create_csr(h_csr.rowptr, h_csr.col, h_csr.val, opts=S.SolveOptions(precision=prec))
    try:
        for sites in ([17], list(range(5, 5 + 33 * 7, 7))):
            B = np.zeros((len(sites), n))
            B[np.arange(len(sites)), sites] = 1.0
            G, used, _ = S.scocg_krylov_sd_multi(h, dev(B), 1, z, np.array(sites)[:, None])
            G = G.cpu().numpy()
            assert np.all(used == 1)
            for r, j in enumerate(sites):
                ref = 1.0 / (z - Hd[j, j])
                assert np.max(np.abs(G[r, 0] - ref)) < 1e-13 * np.max(np.abs(ref)), (prec, j)
    finally:
        S.scocg_destroy(h)
