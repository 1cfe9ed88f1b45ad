"""Continuation of a solve stopped at max_iter (scocg_solve_resume) and its
host checkpoint (scocg_state_save / scocg_state_load), through the C ABI.

The continued solve carries the seed vectors, every shift's recurrence
values and the FP64 seed scalars over from the stopped launch (Sec. III.C's
seed switch reuses its computed information the same way), so with the same
grid it must reproduce the uninterrupted solve bit for bit: G, the freeze
iterations, the residual estimates, the switch count and the final seed.
The uninterrupted solve itself is held to the oracle by the other tests."""
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


def switching_problem():
    """256 rows; the seed z = 30 + i converges first and the solve switches
    seeds (as in the seed-switching parity test)."""
    h = inputs.anderson_csr(4, seed=17)
    b = inputs.random_unit_complex(h.n, 11)
    shifts = np.concatenate([[30.0 + 1.0j], np.linspace(-3, 3, 6) + 0.02j, [-25.0 + 0.5j]])
    return h, b, shifts


def same(info_a, g_a, info_b, g_b):
    assert np.array_equal(g_a, g_b)
    assert np.array_equal(info_a["freeze_iter"], info_b["freeze_iter"])
    assert np.array_equal(info_a["resid"], info_b["resid"])
    for key in ("status", "iters", "n_switch", "seed_final"):
        assert info_a[key] == info_b[key], key


def run_in_pieces(S, h, shifts, rhs, stops, tol, **proj):
    """Solve with max_iter = stops[0], then continue to each next stop, then
    to convergence; every piece but the last ends SCOCG_NOT_CONVERGED."""
    opts = h.opts
    S.scocg_set_opts(h, S.SolveOptions(**{**opts.__dict__, "max_iter": stops[0]}))
    G, info = S.scocg_solve(h, shifts, rhs, tol=tol, **proj)
    assert info["status"] == 1 and info["iters"] == stops[0]
    for nxt in list(stops[1:]) + [0]:
        S.scocg_set_opts(h, S.SolveOptions(**{**opts.__dict__, "max_iter": nxt}))
        G, info = S.scocg_solve_resume(h, shifts, rhs, tol=tol, **proj)
        if nxt:
            assert info["status"] == 1 and info["iters"] == nxt
    return G.cpu().numpy(), info


@pytest.mark.parametrize("prec,layout", [(0, 0), (0, 1), (2, 0), (2, 1), (1, 0)])
def test_resume_equals_uninterrupted_across_switches(S, prec, layout):
    h, b, shifts = switching_problem()
    opts = S.SolveOptions(precision=prec, layout=layout, seed=0)
    tol = 1e-12 if prec != 1 else 1e-5
    hh = S.scocg_create_csr(h.rowptr, h.col, h.val, opts=opts)
    hh.opts = opts
    try:
        bd, cd = cuda(b), cuda(np.conj(b)[None, :])
        G0, info0 = S.scocg_solve(hh, shifts, bd, proj_vec=cd, tol=tol)
        G0 = G0.cpu().numpy()
        assert info0["status"] == 0 and info0["n_switch"] >= 1
        n = info0["iters"]
        for stops in ([3], [n // 3, 2 * n // 3], [n - 1]):
            G1, info1 = run_in_pieces(S, hh, shifts, bd, stops, tol, proj_vec=cd)
            same(info0, G0, info1, G1)
    finally:
        S.scocg_destroy(hh)


def test_resume_without_deferred_shift_update(S):
    """More shifts than 32 per CTA (grid 1, 64 shifts): the shift updates run
    in place rather than inside the next apply; unit projections."""
    h = inputs.anderson_csr(4, seed=5)
    b = inputs.random_unit_complex(h.n, 3)
    shifts = np.linspace(-5, 5, 64) + 0.05j
    opts = S.SolveOptions(precision=2, grid=1)
    hh = S.scocg_create_csr(h.rowptr, h.col, h.val, opts=opts)
    hh.opts = opts
    try:
        bd = cuda(b)
        G0, info0 = S.scocg_solve(hh, shifts, bd, proj_idx=[0, 7], tol=1e-11)
        G0 = G0.cpu().numpy()
        G1, info1 = run_in_pieces(S, hh, shifts, bd, [info0["iters"] // 2], 1e-11, proj_idx=[0, 7])
        same(info0, G0, info1, G1)
    finally:
        S.scocg_destroy(hh)


def test_resume_with_residual_replacement(S):
    """complex64 vectors with the FP64 true-residual replacement every 10
    iterations (shifts near the spectrum, so the seed runs long before any
    switch): the seed direction and compensated solution carry over too."""
    h, b, _ = switching_problem()
    shifts = np.linspace(-3, 3, 6) + 0.02j
    opts = S.SolveOptions(precision=1, replace_every=10)
    hh = S.scocg_create_csr(h.rowptr, h.col, h.val, opts=opts)
    hh.opts = opts
    try:
        bd, cd = cuda(b), cuda(np.conj(b)[None, :])
        G0, info0 = S.scocg_solve(hh, shifts, bd, proj_vec=cd, tol=1e-5)
        G0 = G0.cpu().numpy()
        assert info0["n_replace"] >= 3
        G1, info1 = run_in_pieces(S, hh, shifts, bd, [25], 1e-5, proj_vec=cd)
        same(info0, G0, info1, G1)
        assert info1["n_replace"] == info0["n_replace"]
    finally:
        S.scocg_destroy(hh)


@pytest.mark.parametrize("model", ["ring", "two-orbital"])
def test_resume_hubbard(S, model):
    """Matrix-free handles: the ring (one-pass apply) and the two-orbital
    cluster (two-pass apply), compensated."""
    opts = S.SolveOptions(precision=2)
    if model == "ring":
        hh = S.scocg_create_hubbard(8, 3, 3, 1.0, 4.0, 1.0, True, opts=opts)
        shifts = np.linspace(-4, 12, 24) + 0.1j
    else:
        hh = S.scocg_create_hubbard2(inputs.eg_model(), 2, 2, opts=opts)
        shifts = np.linspace(-12, 48, 24) + 0.1j
    hh.opts = opts
    try:
        n = S.scocg_dim(hh)
        b = inputs.random_unit_complex(n, 4)
        bd, cd = cuda(b), cuda(np.conj(b)[None, :])
        G0, info0 = S.scocg_solve(hh, shifts, bd, proj_vec=cd, tol=1e-10)
        G0 = G0.cpu().numpy()
        G1, info1 = run_in_pieces(S, hh, shifts, bd, [info0["iters"] // 2], 1e-10, proj_vec=cd)
        same(info0, G0, info1, G1)
    finally:
        S.scocg_destroy(hh)


def test_checkpoint_to_host_and_other_handle(S):
    """Stop, save the state to the host, destroy the handle, load the state
    into a new handle of the same H and continue: equal to the uninterrupted
    solve; a state saved from a continuation can be saved again."""
    h, b, shifts = switching_problem()
    opts = S.SolveOptions(precision=2, seed=0)
    bd, cd = cuda(b), cuda(np.conj(b)[None, :])
    h0 = S.scocg_create_csr(h.rowptr, h.col, h.val, opts=opts)
    G0, info0 = S.scocg_solve(h0, shifts, bd, proj_vec=cd, tol=1e-12)
    S.scocg_destroy(h0)
    G0 = G0.cpu().numpy()
    n = info0["iters"]
    h1 = S.scocg_create_csr(h.rowptr, h.col, h.val, opts=S.SolveOptions(precision=2, seed=0, max_iter=n // 3))
    G, info = S.scocg_solve(h1, shifts, bd, proj_vec=cd, tol=1e-12)
    assert info["status"] == 1
    buf = S.scocg_state_save(h1)
    assert buf.size == S.scocg_state_size(h1) > 0
    S.scocg_destroy(h1)
    h2 = S.scocg_create_csr(h.rowptr, h.col, h.val, opts=S.SolveOptions(precision=2, seed=0, max_iter=2 * n // 3))
    try:
        S.scocg_state_load(h2, buf)
        G, info = S.scocg_solve_resume(h2, shifts, bd, proj_vec=cd, tol=1e-12)
        assert info["status"] == 1 and info["iters"] == 2 * n // 3
        buf2 = S.scocg_state_save(h2)
    finally:
        S.scocg_destroy(h2)
    h3 = S.scocg_create_csr(h.rowptr, h.col, h.val, opts=S.SolveOptions(precision=2, seed=0))
    try:
        S.scocg_state_load(h3, buf2)
        G3, info3 = S.scocg_solve_resume(h3, shifts, bd, proj_vec=cd, tol=1e-12)
        same(info0, G0, info3, G3.cpu().numpy())
    finally:
        S.scocg_destroy(h3)


def test_resume_refusals(S):
    h, b, shifts = switching_problem()
    bd, cd = cuda(b), cuda(np.conj(b)[None, :])
    hh = S.scocg_create_csr(h.rowptr, h.col, h.val, opts=S.SolveOptions(precision=2, seed=0, max_iter=5))
    other = S.scocg_create_csr(*(lambda g: (g.rowptr, g.col, g.val))(inputs.anderson_csr(3, seed=1)))
    try:
        # nothing to continue yet
        assert S.scocg_state_size(hh) == 0
        with pytest.raises(S.ScocgError) as e:
            S.scocg_solve_resume(hh, shifts, bd, proj_vec=cd, tol=1e-12)
        assert e.value.code == S.ERR_INVALID
        S.scocg_solve(hh, shifts, bd, proj_vec=cd, tol=1e-12)
        buf = S.scocg_state_save(hh)
        # other shifts, another projection kind, another precision
        for kw in (dict(shifts=shifts[::-1], proj_vec=cd), dict(shifts=shifts, proj_idx=[0])):
            with pytest.raises(S.ScocgError):
                S.scocg_solve_resume(hh, kw.pop("shifts"), bd, tol=1e-12, **kw)
        S.scocg_set_opts(hh, S.SolveOptions(precision=0, seed=0, max_iter=5))
        with pytest.raises(S.ScocgError):
            S.scocg_solve_resume(hh, shifts, bd, proj_vec=cd, tol=1e-12)
        S.scocg_set_opts(hh, S.SolveOptions(precision=2, seed=0))
        # a solve that converges leaves nothing to continue
        S.scocg_solve(hh, shifts, bd, proj_vec=cd, tol=1e-12)
        assert S.scocg_state_size(hh) == 0
        with pytest.raises(S.ScocgError):
            S.scocg_solve_resume(hh, shifts, bd, proj_vec=cd, tol=1e-12)
        # a state does not load into a handle of another H, nor when damaged
        with pytest.raises(S.ScocgError):
            S.scocg_state_load(other, buf)
        bad = buf.copy()
        bad[0] ^= 0xFF
        with pytest.raises(S.ScocgError):
            S.scocg_state_load(hh, bad)
        with pytest.raises(S.ScocgError):
            S.scocg_state_load(hh, buf[: buf.size // 2])
        # several right-hand sides are not continued
        with pytest.raises(ValueError):
            S.scocg_solve_resume(hh, shifts, torch.stack([bd, bd]), proj_vec=cd, tol=1e-12)
    finally:
        S.scocg_destroy(hh)
        S.scocg_destroy(other)
