"""The no-allocation solve (scocg_solve_csr_noalloc) against the handle-based
scocg_solve on the same inputs, through the C ABI.

This entry point serves callers that cannot allocate device memory when they
solve (their memory pool owns the device, or allocation is not allowed in
their loop): it takes the caller's buffers and uses a fixed scratch array
compiled into the library.  This file is collected last on purpose."""
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


def test_no_alloc_matches_handle_solve_twice(S):
    """Two calls in a row (different matrices, shifts and right-hand sides, so
    the second must not see the first's scratch): each equals scocg_solve to
    the FP64 parity tolerance of the other tests (1e-10 relative)."""
    cases = [
        (inputs.anderson_csr(6, seed=5), np.linspace(-5, 5, 40) + 0.05j, 9, "vec"),
        (inputs.chain_csr(1000), np.linspace(-2.5, 2.5, 64) + 0.01j, 3, "idx"),
    ]
    for h, shifts, bseed, proj in cases:
        b = inputs.random_unit_complex(h.n, bseed)
        kw = {"proj_vec": cuda(np.conj(b)[None, :])} if proj == "vec" else {"proj_idx": [0, 7, h.n - 1]}
        hh = S.scocg_create_csr(h.rowptr, h.col, h.val)
        G_ref, info_ref = S.scocg_solve(hh, shifts, cuda(b), tol=1e-12, **kw)
        S.scocg_destroy(hh)
        rp32 = cuda(h.rowptr.astype(np.int32))
        G, info = S.scocg_solve_csr_noalloc(rp32, cuda(h.col), cuda(h.val), shifts, cuda(b), tol=1e-12, **kw)
        assert info["status"] == 0 and info_ref["status"] == 0
        assert relerr(G.cpu().numpy(), G_ref.cpu().numpy()[0]) < 1e-10


def test_no_alloc_rejects_problems_beyond_its_scratch(S):
    h = inputs.chain_csr(2_000_000)
    b = np.zeros(h.n, complex); b[0] = 1
    with pytest.raises(S.ScocgError) as e:
        S.scocg_solve_csr_noalloc(cuda(h.rowptr.astype(np.int32)), cuda(h.col), cuda(h.val), [0.1 + 0.1j], cuda(b),
                                  proj_idx=[0], tol=1e-8)
    assert e.value.code == S.ERR_TOO_LARGE
