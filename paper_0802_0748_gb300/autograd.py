"""torch.autograd.Function over the C-ABI solve and its adjoint.

``shifted_green(val, rowptr, col, shifts, b, proj_idx=..., proj_vec=..., tol=...)``
returns ``G[nproj][nshift]`` (complex128) for the CSR matrix with stored values
``val`` (CUDA float64, may require grad).  Its backward calls ``scocg_grad``:
the adjoint systems are forward solves with the projection vectors as
right-hand sides (``z_k I - H`` is complex symmetric), and

    dL/dval[(a, b)] = Re sum_{k,m} conj(dL/dG_mk) y_mk[a] x_k[b].

Every stored entry is an independent parameter: for a symmetric matrix the
gradient of a symmetric pair is the sum over its two entries.
"""
from __future__ import annotations

import torch

from . import scocg


class ShiftedGreen(torch.autograd.Function):
    @staticmethod
    def forward(ctx, val, rowptr, col, shifts, b, proj_idx, proj_vec, tol, opts):
        h = scocg.scocg_create_csr(rowptr, col, val.detach(), opts=opts)
        try:
            G, info = scocg.scocg_solve(h, shifts, b, proj_idx=proj_idx, proj_vec=proj_vec, tol=tol)
        except Exception:
            scocg.scocg_destroy(h)
            raise
        ctx.h = h
        ctx.args = (shifts, b, proj_idx, proj_vec, tol)
        ctx.info = info
        return G[0]

    @staticmethod
    def backward(ctx, gG):
        shifts, b, proj_idx, proj_vec, tol = ctx.args
        try:
            g, _ = scocg.scocg_grad(ctx.h, shifts, b, gG.contiguous(), proj_idx=proj_idx, proj_vec=proj_vec,
                                    tol=tol)
        finally:
            scocg.scocg_destroy(ctx.h)
            ctx.h = None
        return g, None, None, None, None, None, None, None, None


def shifted_green(val, rowptr, col, shifts, b, proj_idx=None, proj_vec=None, tol=1e-12, opts=None):
    """G[nproj][nshift] = c_m^T (z_k I - H(val))^{-1} b, differentiable in val."""
    return ShiftedGreen.apply(val, rowptr, col, shifts, b, proj_idx, proj_vec, tol, opts)
