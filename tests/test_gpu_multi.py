"""Multi-system launch (many small independent clusters in one cooperative
launch, optionally replayed from a CUDA graph) against the oracle and against
one-system solves, through the C ABI."""
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
    yield scocg
    scocg.scocg_multi_release()


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def relerr(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def clusters(sizes, seed):
    """Anderson clusters of the given linear sizes, each with its own disorder draw."""
    return [inputs.anderson_csr(L, seed=seed + i) for i, L in enumerate(sizes)]


def make_handles(S, hs, prec):
    return [S.scocg_create_csr(h.rowptr, h.col, h.val, opts=S.SolveOptions(precision=prec)) for h in hs]


@pytest.mark.parametrize("prec,bound", [(0, 1e-10), (2, 1e-8)])
def test_multi_matches_oracle(S, oracle_mod, prec, bound):
    """Six clusters of ragged sizes (L = 3..7, 108 to 1372 rows) with different
    shift counts; each system's G against its own oracle solve."""
    hs = clusters([3, 5, 3, 7, 4, 6], seed=300)
    shifts = [np.linspace(-5, 5, 8 + 13 * i) + (0.05 + 0.01 * i) * 1j for i in range(len(hs))]
    rhs = [inputs.random_unit_complex(h.n, 10 + i) for i, h in enumerate(hs)]
    hh = make_handles(S, hs, prec)
    try:
        G, infos = S.scocg_solve_multi(hh, shifts, [cuda(b) for b in rhs], proj_idx=[[0, h.n - 1] for h in hs],
                                       tol=1e-12)
    finally:
        for x in hh:
            S.scocg_destroy(x)
    for s, h in enumerate(hs):
        ref = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts[s], rhs[s], proj_idx=[0, h.n - 1], tol=1e-12)
        assert infos[s]["status"] == 0, s
        assert relerr(G[s].cpu().numpy(), ref.G) < bound, s
        assert infos[s]["resid"].max() <= 1e-12 * (1 + 1e-6)


def test_multi_equals_single_solves_projection_vectors(S):
    """Dense projections: each system's G equals scocg_solve on that system alone."""
    hs = clusters([3, 6, 4], seed=500)
    shifts = [np.linspace(-4, 4, 20) + 0.08j, np.linspace(-6, 6, 33) + 0.03j, np.linspace(-2, 2, 5) + 0.2j]
    rhs = [cuda(inputs.random_unit_complex(h.n, 50 + i)) for i, h in enumerate(hs)]
    pv = [cuda(np.stack([inputs.random_unit_complex(h.n, 70 + i), inputs.random_unit_complex(h.n, 90 + i)]))
          for i, h in enumerate(hs)]
    hh = make_handles(S, hs, 0)
    try:
        G, infos = S.scocg_solve_multi(hh, shifts, rhs, proj_vec=pv, tol=1e-12)
        for s in range(len(hs)):
            g1, i1 = S.scocg_solve(hh[s], shifts[s], rhs[s], proj_vec=pv[s], tol=1e-12)
            assert i1["status"] == 0 and infos[s]["status"] == 0
            assert relerr(G[s].cpu().numpy(), g1.cpu().numpy()) < 1e-10, s
    finally:
        for x in hh:
            S.scocg_destroy(x)


def test_multi_graph_replay_twice_with_new_shifts(S, oracle_mod):
    """use_graph: the first call captures, the second replays with other shift
    values; both agree with the oracle, and a third replay after a one-system
    solve on the same handle (which reuses its workspace) still does."""
    hs = clusters([4, 3, 5, 3], seed=700)
    rhs_np = [inputs.random_unit_complex(h.n, 30 + i) for i, h in enumerate(hs)]
    rhs = [cuda(b) for b in rhs_np]
    proj = [[0] for _ in hs]
    G_out = [torch.zeros((1, 24), dtype=torch.complex128, device="cuda") for _ in hs]
    hh = make_handles(S, hs, 0)
    try:
        for call, (eta, lo) in enumerate([(0.05, -5.0), (0.1, -3.0), (0.07, -4.0)]):
            shifts = [np.linspace(lo, -lo, 24) + eta * 1j for _ in hs]
            if call == 2:
                S.scocg_solve(hh[1], shifts[1], rhs[1], proj_idx=[0], tol=1e-12)
            G, infos = S.scocg_solve_multi(hh, shifts, rhs, proj_idx=proj, tol=1e-12, use_graph=True, G_out=G_out)
            for s, h in enumerate(hs):
                ref = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts[s], rhs_np[s], proj_idx=[0], tol=1e-12)
                assert infos[s]["status"] == 0, (call, s)
                assert relerr(G[s].cpu().numpy(), ref.G) < 1e-10, (call, s)
    finally:
        S.scocg_multi_release()
        for x in hh:
            S.scocg_destroy(x)


def test_multi_many_clusters_uneven(S, oracle_mod):
    """The cluster work list's shape: 96 Anderson clusters of uneven edge length
    (L = 3..12, 108 to 6,912 rows, a bounded sample), 64 shifts each, unit
    projection on site 0; eight systems checked against the oracle, all against
    the tolerance."""
    Ls = inputs.cluster_sizes(96, 3, 12, seed=11)
    hs = [inputs.anderson_csr(int(L), seed=900 + i) for i, L in enumerate(Ls)]
    shifts = [np.linspace(-6.5, 6.5, 64) + 0.05j for _ in hs]
    rhs_np = [np.eye(1, h.n, 0, dtype=np.complex128)[0] for h in hs]
    hh = make_handles(S, hs, 0)
    try:
        G, infos = S.scocg_solve_multi(hh, shifts, [cuda(b) for b in rhs_np], proj_idx=[[0]] * len(hs), tol=1e-10)
    finally:
        for x in hh:
            S.scocg_destroy(x)
    assert all(i["status"] == 0 for i in infos)
    assert all(i["resid"].max() <= 1e-10 * (1 + 1e-6) for i in infos)
    for s in np.random.default_rng(11).choice(len(hs), size=8, replace=False):
        h = hs[s]
        ref = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts[s], rhs_np[s], proj_idx=[0], tol=1e-10)
        assert relerr(G[s].cpu().numpy(), ref.G) < 1e-7, s


def test_multi_invalid(S):
    hs = clusters([3, 4], seed=1)
    hh = make_handles(S, hs, 0)
    h_df = S.scocg_create_csr(hs[0].rowptr, hs[0].col, hs[0].val, opts=S.SolveOptions(precision=2))
    z = [np.array([0.1j]), np.array([0.1j])]
    b = [cuda(np.ones(h.n, complex)) for h in hs]
    try:
        with pytest.raises(RuntimeError):   # the same handle twice
            S.scocg_solve_multi([hh[0], hh[0]], z, [b[0], b[0]], proj_idx=[[0], [0]])
        with pytest.raises(RuntimeError):   # mixed precisions
            S.scocg_solve_multi([hh[0], h_df], z, [b[0], b[0]], proj_idx=[[0], [0]])
        with pytest.raises(RuntimeError):   # projection index out of range
            S.scocg_solve_multi(hh, z, b, proj_idx=[[0], [hs[1].n]])
        hc = S.scocg_create_csr(*[getattr(inputs.chain_csr(50), f) for f in ("rowptr", "col", "val")])
        try:   # different device layouts (blocked and CSR) cannot share a launch
            with pytest.raises(RuntimeError):
                S.scocg_solve_multi([hh[0], hc], z, [b[0], cuda(np.ones(50, complex))], proj_idx=[[0], [0]])
        finally:
            S.scocg_destroy(hc)
    finally:
        for x in hh + [h_df]:
            S.scocg_destroy(x)
