"""The no-allocation solve (scocg_solve_csr_noalloc) against the handle-based
scocg_solve on the same inputs, through the C ABI.

This entry point serves callers that cannot allocate device memory when they
solve (their memory pool owns the device, or allocation is not allowed in
their loop): it takes the caller's buffers and uses a fixed scratch array
compiled into the library.  This file is collected last on purpose."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_0802_0748_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def handle_solve(S, h, shifts, b, tol, **kw):
    hh = S.scocg_create_csr(h.rowptr, h.col, h.val)
    try:
        G, info = S.scocg_solve(hh, shifts, cuda(b), tol=tol, **kw)
    finally:
        S.scocg_destroy(hh)
    return G.cpu().numpy()[0], info


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
        G_ref, info_ref = handle_solve(S, h, shifts, b, 1e-12, **kw)
        rp32 = cuda(h.rowptr.astype(np.int32))
        G, info = S.scocg_solve_csr_noalloc(rp32, cuda(h.col), cuda(h.val), shifts, cuda(b), tol=1e-12, **kw)
        assert info["status"] == 0 and info_ref["status"] == 0
        assert relerr(G.cpu().numpy(), G_ref) < 1e-10


def test_no_alloc_allocates_nothing_near_its_limit(S):
    """A problem just under the scratch limit (780,000-row chain: about
    32 n bytes of vectors in the 24 MiB array) with the output buffer passed
    in: after a first call, a second call leaves both torch's reserved memory
    and the device's free memory (cudaMemGetInfo) unchanged, and both calls
    equal the handle solve to 1e-10."""
    h = inputs.chain_csr(780_000)
    shifts = np.linspace(-2.5, 2.5, 16) + 0.1j
    b = np.zeros(h.n, complex); b[0] = 1.0
    G_ref, _ = handle_solve(S, h, shifts, b, 1e-12, proj_idx=[0, 5])
    rp32, col, val, bb = cuda(h.rowptr.astype(np.int32)), cuda(h.col), cuda(h.val), cuda(b)
    G_out = torch.zeros((2, shifts.size), dtype=torch.complex128, device="cuda")
    G1, info1 = S.scocg_solve_csr_noalloc(rp32, col, val, shifts, bb, proj_idx=[0, 5], tol=1e-12, G_out=G_out)
    g1 = G1.cpu().numpy()
    torch.cuda.synchronize()
    reserved = torch.cuda.memory_reserved()
    free0, _ = torch.cuda.mem_get_info()
    G_out.zero_()
    G2, info2 = S.scocg_solve_csr_noalloc(rp32, col, val, shifts, bb, proj_idx=[0, 5], tol=1e-12, G_out=G_out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_reserved() == reserved
    assert free1 == free0
    assert G2.data_ptr() == G_out.data_ptr()
    assert info1["status"] == 0 and info2["status"] == 0
    assert relerr(g1, G_ref) < 1e-10
    assert relerr(G2.cpu().numpy(), G_ref) < 1e-10


def test_no_alloc_rejects_problems_beyond_its_scratch(S):
    h = inputs.chain_csr(2_000_000)
    b = np.zeros(h.n, complex); b[0] = 1
    with pytest.raises(S.ScocgError) as e:
        S.scocg_solve_csr_noalloc(cuda(h.rowptr.astype(np.int32)), cuda(h.col), cuda(h.val), [0.1 + 0.1j], cuda(b),
                                  proj_idx=[0], tol=1e-8)
    assert e.value.code == S.ERR_TOO_LARGE


CHECKED_SCRIPT = r"""
import numpy as np, torch
from paper_0802_0748_gb300 import build, inputs
build.build(checked=True)
from paper_0802_0748_gb300 import scocg as S
assert str(S.LIB_PATH).endswith("checked/libscocg.so")
h = inputs.chain_csr(200)
col = h.col.copy()
col[37] = h.n + 11          # out of range: the checked kernel records it and skips the load
b = np.zeros(h.n, complex); b[0] = 1.0
try:
    S.scocg_solve_csr_noalloc(torch.from_numpy(h.rowptr.astype(np.int32)).cuda(), torch.from_numpy(col).cuda(),
                              torch.from_numpy(h.val).cuda(), [0.3 + 0.1j], torch.from_numpy(b).cuda(),
                              proj_idx=[0], tol=1e-10)
except S.ScocgError as e:
    assert e.code == S.ERR_INVALID, e.code
    print("rejected")
"""


def test_no_alloc_checked_build_reports_a_bad_column(S):
    """In the bounds-checked build an out-of-range column index of the caller's
    CSR is recorded and skipped by the kernel (no access outside the buffers),
    and the call returns SCOCG_ERR_INVALID."""
    env = dict(os.environ, SCOCG_LIB="checked")
    r = subprocess.run([sys.executable, "-c", CHECKED_SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "rejected" in r.stdout
