"""Full-size parity of the batched and matrix-free workloads in the launch
configuration bench.py times, on sampled outputs the oracle can compute one by
one.  Every comparison stops both sides after the same number of seed
iterations, before any Ritz value converges (after that the short recurrences
lose orthogonality and unconverged iterates depend on rounding order), so the
two sides compute the same iterate:

* block mode (32^3 x 4 Anderson, 131,072 rows, 256 unit right-hand sides x
  256 shifts, compensated FP32, autotuned slot count): 4 sampled right-hand
  sides x 12 sampled shifts;
* the multi-system launch (32 clusters of edge 14..50, 5,118,460 rows,
  compensated FP32, graph replay): 3 sampled clusters x 8 shifts;
* the 14-site Hubbard ring (11,778,624 states), compensated FP32 and FP64:
  8 sampled shifts (the oracle solves on the CSR it builds from the literal
  Jordan-Wigner definition).

Compensated FP32 against the FP64 oracle: relative 1e-9 after 12-30
iterations of ~1e6-1e7-term sums."""
import numpy as np
import pytest

from paper_0802_0748_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BATCH_BOUNDS = inputs.BATCH32_BOUNDS


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


def test_batch_full_size_block_mode(S, oracle_mod):
    wl = inputs.workload("batch", "full", bounds=BATCH_BOUNDS)
    h = wl.csr
    n_it = 30
    hh = S.scocg_create_csr(h.rowptr, h.col, h.val,
                            opts=S.SolveOptions(precision=S.MIXED_DF, autotune=1, max_iter=n_it))
    try:
        G, info = S.scocg_solve(hh, wl.shifts, cuda(wl.rhs), proj_idx=wl.proj_idx, tol=0.0)
    finally:
        S.scocg_destroy(hh)
    assert info["status"] == 1          # capped: every right-hand side ran n_it iterations
    G = G.cpu().numpy()
    seed = oracle_mod.default_seed(wl.shifts)
    ks = np.unique(np.concatenate([[seed], np.linspace(0, wl.shifts.size - 1, 11).astype(int)]))
    for j in (0, 77, 150, 255):
        ref = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, wl.shifts[ks], wl.rhs[j],
                                      proj_idx=[int(wl.proj_idx[j, 0])], tol=0.0, max_iter=n_it,
                                      seed=int(np.where(ks == seed)[0][0]))
        assert relerr(G[j][:, ks], ref.G) < 1e-9, j


def test_clusters_full_size_multi_launch(S, oracle_mod):
    Ls = inputs.cluster_sizes(32, 14, 50, seed=31)
    hs = [inputs.anderson_csr(int(L), seed=3100 + i) for i, L in enumerate(Ls)]
    shifts = [np.linspace(-6.5, 6.5, 128) + 1e-2j for _ in hs]
    b = [inputs.random_unit_complex(h.n, 3200 + i) for i, h in enumerate(hs)]
    n_it = 20
    hh = [S.scocg_create_csr(h.rowptr, h.col, h.val, opts=S.SolveOptions(precision=S.MIXED_DF, max_iter=n_it))
          for h in hs]
    G_out = [torch.zeros((1, 128), dtype=torch.complex128, device="cuda") for _ in hs]
    try:
        G, infos = S.scocg_solve_multi(hh, shifts, [cuda(x) for x in b],
                                       proj_vec=[cuda(np.conj(x)[None, :]) for x in b], tol=0.0, use_graph=True,
                                       G_out=G_out)
    finally:
        S.scocg_multi_release()
        for x in hh:
            S.scocg_destroy(x)
    seed = oracle_mod.default_seed(shifts[0])
    ks = np.unique(np.concatenate([[seed], np.linspace(0, 127, 7).astype(int)]))
    for s in (int(np.argmax(Ls)), int(np.argmin(Ls)), 5):
        h = hs[s]
        ref = oracle_mod.shifted_cocg(h.rowptr, h.col, h.val, shifts[s][ks], b[s], proj_vec=[np.conj(b[s])],
                                      tol=0.0, max_iter=n_it, seed=int(np.where(ks == seed)[0][0]))
        assert relerr(G[s].cpu().numpy()[:, ks], ref.G) < 1e-9, (s, int(Ls[s]))


@pytest.mark.parametrize("prec,bound", [(0, 1e-10), (2, 1e-9)])
def test_hubbard_full_size_solve(S, oracle_mod, prec, bound):
    wl = inputs.workload("hubbard", "full")
    p = wl.hubbard
    n_it = 12
    hh = S.scocg_create_hubbard(p["L"], p["n_up"], p["n_dn"], p["t"], p["U"], p["V"], p["periodic"],
                                opts=S.SolveOptions(precision=prec, max_iter=n_it))
    try:
        G, info = S.scocg_solve(hh, wl.shifts, cuda(wl.rhs[0]), proj_vec=cuda(wl.proj_vec), tol=0.0)
    finally:
        S.scocg_destroy(hh)
    G = G.cpu().numpy()[0]
    rp, c, v = oracle_mod.hubbard_csr(p["L"], p["n_up"], p["n_dn"], p["t"], p["U"], p["V"], p["periodic"])
    seed = oracle_mod.default_seed(wl.shifts)
    ks = np.unique(np.concatenate([[seed], np.linspace(0, 127, 7).astype(int)]))
    ref = oracle_mod.shifted_cocg(rp, c, v, wl.shifts[ks], wl.rhs[0], proj_vec=wl.proj_vec, tol=0.0,
                                  max_iter=n_it, seed=int(np.where(ks == seed)[0][0]))
    assert relerr(G[:, ks], ref.G) < bound
