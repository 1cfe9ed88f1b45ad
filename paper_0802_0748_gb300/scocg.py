"""Thin ctypes binding of the C ABI in include/scocg.h (same entry-point names).

Only argument marshalling happens here: device buffers are PyTorch CUDA
tensors, host arrays are numpy arrays, and every step of the solve runs in the
CUDA library.  There is no CPU fallback: if the library is missing, loading it
raises.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from pathlib import Path

import numpy as np

import os

# SCOCG_LIB=checked selects the bounds-checked build (see build.py)
_variant = os.environ.get("SCOCG_LIB", "")
LIB_PATH = Path(__file__).resolve().parent / "_build" / (
    f"{_variant}/libscocg.so" if _variant else "libscocg.so")

OK, NOT_CONVERGED = 0, 1
ERR_INVALID, ERR_CUDA, ERR_OOM, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_UNSYMMETRIC, ERR_TOO_LARGE = -1, -2, -3, -4, -5, -6, -7
FP64, MIXED, MIXED_DF = 0, 1, 2

EXPORTED = [
    "scocg_create_csr", "scocg_create_hubbard", "scocg_dim", "scocg_set_opts", "scocg_apply",
    "scocg_solve", "scocg_solve_full", "scocg_grad", "scocg_destroy", "scocg_strerror",
    "scocg_hubbard_tables", "scocg_solve_csr_noalloc", "scocg_solve_multi", "scocg_multi_release",
    "scocg_density", "scocg_ground_state", "scocg_excite", "scocg_krylov_sd", "scocg_create_hubbard2",
    "scocg_solve_resume", "scocg_state_size", "scocg_state_save", "scocg_state_load", "scocg_krylov_sd_multi",
]


class ScocgError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {strerror(code)} ({code})")
        self.code = code


class c128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_iter", ctypes.c_int), ("replace_every", ctypes.c_int),
                ("seed", ctypes.c_int), ("no_switch", ctypes.c_int), ("autotune", ctypes.c_int),
                ("timeout_ms", ctypes.c_double), ("layout", ctypes.c_int), ("grid", ctypes.c_int),
                ("debug_inject", ctypes.c_int), ("rhs_tile", ctypes.c_int)]


class GroundInfo(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("lanczos_steps", ctypes.c_longlong), ("cg_steps", ctypes.c_longlong),
                ("residual", ctypes.c_double), ("seconds", ctypes.c_double), ("bytes_per_step", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("n_switch", ctypes.c_int), ("seed_final", ctypes.c_int),
                ("n_replace", ctypes.c_int), ("shift_iters", ctypes.c_longlong),
                ("freeze_iter", ctypes.POINTER(ctypes.c_int)), ("resid", ctypes.POINTER(ctypes.c_double)),
                ("seconds", ctypes.c_double), ("bytes_per_iter", ctypes.c_double)]


@dataclass
class SolveOptions:
    precision: int = FP64
    max_iter: int = 0
    replace_every: int = 0
    seed: int = -1
    no_switch: int = 0
    autotune: int = 0
    timeout_ms: float = 0.0
    layout: int = 0
    grid: int = 0
    debug_inject: int = 0
    rhs_tile: int = 0

    def c(self) -> Opts:
        return Opts(self.precision, self.max_iter, self.replace_every, self.seed, self.no_switch,
                    self.autotune, self.timeout_ms, self.layout, self.grid, self.debug_inject, self.rhs_tile)


_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(str(LIB_PATH))
        P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        D = ctypes.c_double
        L.scocg_create_csr.argtypes = [ctypes.POINTER(P), I64, I64, P, P, P, I, ctypes.POINTER(Opts), P]
        L.scocg_create_hubbard.argtypes = [ctypes.POINTER(P), I, I, I, D, D, D, I, ctypes.POINTER(Opts), P]
        L.scocg_create_hubbard2.argtypes = [ctypes.POINTER(P), I, I, P, P, P, D, D, D, D, D, I, I,
                                            ctypes.POINTER(Opts), P]
        L.scocg_dim.argtypes = [P, ctypes.POINTER(I64)]
        L.scocg_set_opts.argtypes = [P, ctypes.POINTER(Opts)]
        L.scocg_apply.argtypes = [P, c128, P, P, I]
        L.scocg_solve.argtypes = [P, P, I, P, I, P, P, I, D, P, ctypes.POINTER(Info)]
        L.scocg_solve_resume.argtypes = [P, P, I, P, P, P, I, D, P, ctypes.POINTER(Info)]
        L.scocg_state_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.scocg_state_save.argtypes = [P, P, ctypes.c_size_t]
        L.scocg_state_load.argtypes = [P, P, ctypes.c_size_t]
        L.scocg_solve_full.argtypes = [P, P, I, P, D, P, ctypes.POINTER(Info)]
        L.scocg_grad.argtypes = [P, P, I, P, I, P, P, I, D, P, P, ctypes.POINTER(Info)]
        L.scocg_density.argtypes = [P, D, D, D, D, D, I, P, I, P, P, I, D, P, ctypes.POINTER(Info)]
        L.scocg_ground_state.argtypes = [P, P, P, I, I, I, D, ctypes.POINTER(D), ctypes.POINTER(GroundInfo)]
        L.scocg_excite.argtypes = [P, P, I, I, I, P, P]
        L.scocg_krylov_sd.argtypes = [P, P, I, P, I, P, P, I, P, P, P, ctypes.POINTER(I), ctypes.POINTER(D)]
        L.scocg_krylov_sd_multi.argtypes = [P, P, I, I, P, I, P, I, P, P, ctypes.POINTER(D)]
        L.scocg_destroy.argtypes = [P]
        L.scocg_destroy.restype = None
        L.scocg_strerror.argtypes = [I]
        L.scocg_strerror.restype = ctypes.c_char_p
        L.scocg_hubbard_tables.argtypes = [P, I, ctypes.POINTER(ctypes.c_int32), P, P, P]
        L.scocg_solve_csr_noalloc.argtypes = [I64, I64, P, P, P, P, I, P, P, P, I, D, I, P,
                                              ctypes.POINTER(Info), P]
        L.scocg_solve_multi.argtypes = [I, P, P, P, P, P, P, P, D, P, P, I]
        L.scocg_multi_release.argtypes = []
        L.scocg_multi_release.restype = None
        for name in EXPORTED:
            if name not in ("scocg_destroy", "scocg_strerror", "scocg_multi_release"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().scocg_strerror(code).decode()


def _check(code: int, where: str) -> int:
    if code < 0:
        raise ScocgError(code, where)
    return code


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t):
    return ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, numel: int | None, name: str):
    """Checks that a device argument is a contiguous CUDA tensor of the given
    dtype and element count (the C side reads exactly that many elements)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, not {t.numel()}")
    return t


def _handle_n(h) -> int:
    n = getattr(h, "n", None)
    return int(n) if n is not None else scocg_dim(h)


class Handle:
    """Owns one scocg_handle; destroyed by close() or garbage collection."""

    def __init__(self, ptr: ctypes.c_void_p, stream):
        self._ptr = ptr
        self.stream = stream

    @property
    def ptr(self):
        if self._ptr is None:
            raise ValueError("handle closed")
        return self._ptr

    def close(self):
        if self._ptr is not None and _lib is not None:
            _lib.scocg_destroy(self._ptr)
        self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def scocg_create_csr(rowptr, col, val, opts: SolveOptions | None = None, stream=None) -> Handle:
    """scocg_create_csr: H from CSR arrays (numpy on the host, or torch CUDA tensors)."""
    import torch
    out = ctypes.c_void_p()
    o = (opts or SolveOptions()).c()
    if isinstance(rowptr, torch.Tensor):
        rp = rowptr.to(torch.int64).contiguous(); cc = col.to(torch.int32).contiguous()
        vv = val.to(torch.float64).contiguous()
        n, nnz = rp.numel() - 1, cc.numel()
        code = lib().scocg_create_csr(ctypes.byref(out), n, nnz, _dev(rp), _dev(cc), _dev(vv), 1,
                                      ctypes.byref(o), _stream_ptr(stream))
    else:
        rp = np.ascontiguousarray(rowptr, dtype=np.int64); cc = np.ascontiguousarray(col, dtype=np.int32)
        vv = np.ascontiguousarray(val, dtype=np.float64)
        n, nnz = rp.size - 1, cc.size
        code = lib().scocg_create_csr(ctypes.byref(out), n, nnz, rp.ctypes.data, cc.ctypes.data,
                                      vv.ctypes.data, 0, ctypes.byref(o), _stream_ptr(stream))
    _check(code, "scocg_create_csr")
    h = Handle(out, stream)
    h.n, h.nnz = n, nnz
    return h


def scocg_create_hubbard(L, n_up, n_dn, t, U, V, periodic=True, opts: SolveOptions | None = None,
                         stream=None) -> Handle:
    """scocg_create_hubbard: matrix-free extended Hubbard ring (Sec. IV.B)."""
    out = ctypes.c_void_p()
    o = (opts or SolveOptions()).c()
    code = lib().scocg_create_hubbard(ctypes.byref(out), L, n_up, n_dn, t, U, V, int(bool(periodic)),
                                      ctypes.byref(o), _stream_ptr(stream))
    _check(code, "scocg_create_hubbard")
    h = Handle(out, stream)
    h.L = L
    h.sector = (int(n_up), int(n_dn))
    return h


def scocg_create_hubbard2(model: dict, n_up: int, n_dn: int, opts: SolveOptions | None = None,
                          stream=None) -> Handle:
    """scocg_create_hubbard2: matrix-free two-orbital extended Hubbard model
    (Sec. IV.B).  model: dict with n_sites, bonds [(i, j)], bond_t [nb][2][2],
    U, Up, J, Jp, V."""
    out = ctypes.c_void_p()
    o = (opts or SolveOptions()).c()
    bi = np.ascontiguousarray([b[0] for b in model["bonds"]], dtype=np.int32)
    bj = np.ascontiguousarray([b[1] for b in model["bonds"]], dtype=np.int32)
    bt = np.ascontiguousarray(model["bond_t"], dtype=np.float64).reshape(-1, 2, 2)
    if bt.shape[0] != bi.size:
        raise ValueError("bond_t must hold one 2x2 block per bond")
    code = lib().scocg_create_hubbard2(ctypes.byref(out), int(model["n_sites"]), int(bi.size), bi.ctypes.data,
                                       bj.ctypes.data, bt.ctypes.data, float(model["U"]), float(model["Up"]),
                                       float(model["J"]), float(model["Jp"]), float(model["V"]), int(n_up), int(n_dn),
                                       ctypes.byref(o), _stream_ptr(stream))
    _check(code, "scocg_create_hubbard2")
    h = Handle(out, stream)
    h.L = 2 * int(model["n_sites"])
    h.sector = (int(n_up), int(n_dn))
    return h


def scocg_dim(h: Handle) -> int:
    n = ctypes.c_int64()
    _check(lib().scocg_dim(h.ptr, ctypes.byref(n)), "scocg_dim")
    return int(n.value)


def scocg_set_opts(h: Handle, opts: SolveOptions) -> None:
    o = opts.c()
    _check(lib().scocg_set_opts(h.ptr, ctypes.byref(o)), "scocg_set_opts")


def scocg_apply(h: Handle, z: complex, x, precision: int = FP64):
    """y = (z I - H) x; x is a CUDA complex128 (FP64), complex64 (MIXED) or
    float32 [N, 4] {re.hi, im.hi, re.lo, im.lo} (MIXED_DF) tensor."""
    import torch
    want = {FP64: torch.complex128, MIXED: torch.complex64, MIXED_DF: torch.float32}[precision]
    if x.dtype != want or not x.is_cuda or (precision == MIXED_DF and x.shape[-1] != 4):
        raise TypeError(f"x must be a CUDA {want} tensor" + (" of shape [N, 4]" if precision == MIXED_DF else ""))
    x = x.contiguous()
    y = torch.empty_like(x)
    _check(lib().scocg_apply(h.ptr, c128(float(np.real(z)), float(np.imag(z))), _dev(x), _dev(y), precision),
           "scocg_apply")
    return y


def _shifts(shifts):
    z = np.ascontiguousarray(np.asarray(shifts, dtype=np.complex128))
    return z, z.ctypes.data


def _info_struct(nrhs, nshift):
    it = np.zeros(nrhs * nshift, dtype=np.int32)
    rs = np.zeros(nrhs * nshift, dtype=np.float64)
    info = Info()
    info.freeze_iter = it.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    info.resid = rs.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return info, it, rs


def _info_dict(info, it, rs, nrhs, nshift, status):
    return {"status": status, "iters": info.iters, "n_switch": info.n_switch, "seed_final": info.seed_final,
            "n_replace": info.n_replace, "shift_iters": int(info.shift_iters), "seconds": info.seconds,
            "bytes_per_iter": info.bytes_per_iter, "freeze_iter": it.reshape(nrhs, nshift),
            "resid": rs.reshape(nrhs, nshift)}


def scocg_solve(h: Handle, shifts, rhs, proj_idx=None, proj_vec=None, tol: float = 1e-10):
    """scocg_solve: returns (G [nrhs][nproj][nshift] CUDA complex128 tensor, info dict).

    rhs: CUDA complex128 [nrhs][N] (or [N]); proj_idx: host int [nrhs][nproj]
    (or [nproj], shared); proj_vec: CUDA complex128 [nproj][N]."""
    return _solve(h, shifts, rhs, proj_idx, proj_vec, tol, resume=False)


def scocg_solve_resume(h: Handle, shifts, rhs, proj_idx=None, proj_vec=None, tol: float = 1e-10):
    """scocg_solve_resume: continues the handle's last solve, stopped at
    max_iter, with the same arguments (one right-hand side); returns what
    scocg_solve returns."""
    return _solve(h, shifts, rhs, proj_idx, proj_vec, tol, resume=True)


def scocg_state_size(h: Handle) -> int:
    """Bytes of the handle's continuation state (0 when there is none)."""
    n = ctypes.c_size_t(0)
    lib().scocg_state_size(h.ptr, ctypes.byref(n))
    return int(n.value)


def scocg_state_save(h: Handle) -> np.ndarray:
    """The continuation state of the handle's last stopped solve as a host uint8 array."""
    n = ctypes.c_size_t(0)
    _check(lib().scocg_state_size(h.ptr, ctypes.byref(n)), "scocg_state_size")
    buf = np.empty(n.value, dtype=np.uint8)
    _check(lib().scocg_state_save(h.ptr, buf.ctypes.data, buf.size), "scocg_state_save")
    return buf


def scocg_state_load(h: Handle, buf) -> None:
    """Makes a saved state the handle's continuation state (scocg_solve_resume continues it)."""
    b = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().scocg_state_load(h.ptr, b.ctypes.data, b.size), "scocg_state_load")


def _solve(h: Handle, shifts, rhs, proj_idx, proj_vec, tol, resume: bool):
    import torch
    z, zp = _shifts(shifts)
    K = z.size
    n = _handle_n(h)
    rhs = rhs if rhs.dim() == 2 else rhs.reshape(1, -1)
    if rhs.dtype != torch.complex128 or not rhs.is_cuda:
        raise TypeError("rhs must be a CUDA complex128 tensor")
    rhs = rhs.contiguous()
    nrhs = rhs.shape[0]
    _need(rhs, torch.complex128, nrhs * n, "rhs")
    pidx_p = pvec_p = None
    if proj_idx is not None:
        pidx = np.ascontiguousarray(np.asarray(proj_idx, dtype=np.int64))
        if pidx.ndim == 1:
            pidx = np.ascontiguousarray(np.broadcast_to(pidx, (nrhs, pidx.size)))
        M = pidx.shape[1]
        pidx_p = pidx.ctypes.data
    else:
        pv = proj_vec if proj_vec.dim() == 2 else proj_vec.reshape(1, -1)
        if pv.dtype != torch.complex128 or not pv.is_cuda:
            raise TypeError("proj_vec must be a CUDA complex128 tensor")
        pv = pv.contiguous()
        M = pv.shape[0]
        _need(pv, torch.complex128, M * n, "proj_vec")
        pvec_p = _dev(pv)
    G = torch.zeros((nrhs, M, K), dtype=torch.complex128, device=rhs.device)
    info, it, rs = _info_struct(nrhs, K)
    if resume:
        if nrhs != 1:
            raise ValueError("scocg_solve_resume continues one right-hand side")
        code = lib().scocg_solve_resume(h.ptr, zp, K, _dev(rhs), pidx_p, pvec_p, M, float(tol), _dev(G),
                                        ctypes.byref(info))
        _check(code, "scocg_solve_resume")
    else:
        code = lib().scocg_solve(h.ptr, zp, K, _dev(rhs), nrhs, pidx_p, pvec_p, M, float(tol), _dev(G),
                                 ctypes.byref(info))
        _check(code, "scocg_solve")
    return G, _info_dict(info, it, rs, nrhs, K, code)


def scocg_density(h: Handle, mu: float, kT: float, delta: float, emin: float, emax: float, nquad: int, rhs,
                  proj_idx=None, proj_vec=None, tol: float = 1e-10):
    """scocg_density: returns (rho [nrhs][nproj] CUDA float64 tensor, info dict).

    rhs / proj_idx / proj_vec as in scocg_solve; the shifts are the nquad grid
    energies of [emin, emax] plus i delta."""
    import torch
    n = _handle_n(h)
    rhs = rhs if rhs.dim() == 2 else rhs.reshape(1, -1)
    if rhs.dtype != torch.complex128 or not rhs.is_cuda:
        raise TypeError("rhs must be a CUDA complex128 tensor")
    rhs = rhs.contiguous()
    nrhs = rhs.shape[0]
    _need(rhs, torch.complex128, nrhs * n, "rhs")
    pidx_p = pvec_p = None
    keep = None
    if proj_idx is not None:
        keep = np.ascontiguousarray(np.asarray(proj_idx, dtype=np.int64))
        if keep.ndim == 1:
            keep = np.ascontiguousarray(np.broadcast_to(keep, (nrhs, keep.size)))
        M = keep.shape[1]
        pidx_p = keep.ctypes.data
    else:
        pv = (proj_vec if proj_vec.dim() == 2 else proj_vec.reshape(1, -1)).contiguous()
        if pv.dtype != torch.complex128 or not pv.is_cuda:
            raise TypeError("proj_vec must be a CUDA complex128 tensor")
        keep = pv
        M = pv.shape[0]
        _need(pv, torch.complex128, M * n, "proj_vec")
        pvec_p = _dev(pv)
    rho = torch.zeros((nrhs, M), dtype=torch.float64, device=rhs.device)
    info, it, rs = _info_struct(nrhs, int(nquad))
    code = lib().scocg_density(h.ptr, float(mu), float(kT), float(delta), float(emin), float(emax), int(nquad),
                               _dev(rhs), nrhs, pidx_p, pvec_p, M, float(tol), _dev(rho), ctypes.byref(info))
    _check(code, "scocg_density")
    return rho, _info_dict(info, it, rs, nrhs, int(nquad), code)


def scocg_solve_full(h: Handle, shifts, rhs, tol: float = 1e-10):
    """scocg_solve_full: returns (X [nshift][N] CUDA complex128 tensor, info dict)."""
    import torch
    z, zp = _shifts(shifts)
    K = z.size
    rhs = _need(rhs.reshape(-1).contiguous(), torch.complex128, _handle_n(h), "rhs")
    X = torch.zeros((K, rhs.numel()), dtype=torch.complex128, device=rhs.device)
    info, it, rs = _info_struct(1, K)
    code = lib().scocg_solve_full(h.ptr, zp, K, _dev(rhs), float(tol), _dev(X), ctypes.byref(info))
    _check(code, "scocg_solve_full")
    return X, _info_dict(info, it, rs, 1, K, code)


def scocg_grad(h: Handle, shifts, rhs, dL_dG, proj_idx=None, proj_vec=None, tol: float = 1e-10):
    """scocg_grad: returns (dL/dval CUDA float64 [nnz], info dict)."""
    import torch
    z, zp = _shifts(shifts)
    K = z.size
    n = _handle_n(h)
    rhs = _need(rhs.reshape(1, -1).contiguous(), torch.complex128, n, "rhs")
    pidx_p = pvec_p = None
    if proj_idx is not None:
        pidx = np.ascontiguousarray(np.asarray(proj_idx, dtype=np.int64).reshape(1, -1))
        M = pidx.shape[1]
        pidx_p = pidx.ctypes.data
    else:
        pv = (proj_vec if proj_vec.dim() == 2 else proj_vec.reshape(1, -1)).contiguous()
        M = pv.shape[0]
        _need(pv, torch.complex128, M * n, "proj_vec")
        pvec_p = _dev(pv)
    g = _need(dL_dG.to(torch.complex128).contiguous(), torch.complex128, M * K, "dL_dG")
    out = torch.zeros(int(h.nnz), dtype=torch.float64, device=rhs.device)
    info, it, rs = _info_struct(1, K)
    code = lib().scocg_grad(h.ptr, zp, K, _dev(rhs), 1, pidx_p, pvec_p, M, float(tol), _dev(g), _dev(out),
                            ctypes.byref(info))
    _check(code, "scocg_grad")
    return out, _info_dict(info, it, rs, 1, K, code)


def scocg_destroy(h: Handle) -> None:
    h.close()


def scocg_strerror(code: int) -> str:
    return strerror(code)


def scocg_ground_state(h: Handle, v0, m: int = 60, cg_steps: int = 0, max_cycles: int = 50, tol: float = 1e-10):
    """scocg_ground_state: returns (E, psi CUDA float64 [N], info dict).

    v0: CUDA float64 [N] start vector.  Lanczos / CG-inverse-iteration cycles
    (Sec. II.B) until ||H psi - E psi|| <= tol."""
    import torch
    if v0.dtype != torch.float64 or not v0.is_cuda:
        raise TypeError("v0 must be a CUDA float64 tensor")
    if v0.numel() != scocg_dim(h):
        raise ValueError("v0 must have the handle's dimension")
    v0 = v0.reshape(-1).contiguous()
    psi = torch.empty_like(v0)
    E = ctypes.c_double()
    info = GroundInfo()
    code = lib().scocg_ground_state(h.ptr, _dev(v0), _dev(psi), int(m), int(cg_steps), int(max_cycles), float(tol),
                                    ctypes.byref(E), ctypes.byref(info))
    _check(code, "scocg_ground_state")
    return E.value, psi, {"status": code, "cycles": info.cycles, "lanczos_steps": int(info.lanczos_steps),
                          "cg_steps": int(info.cg_steps), "residual": info.residual, "seconds": info.seconds,
                          "bytes_per_step": info.bytes_per_step}


def scocg_krylov_sd_multi(h: Handle, B, nu: int, shifts, proj_idx):
    """scocg_krylov_sd_multi: returns (G [nrhs][nproj][nshift] CUDA complex128,
    nu_used int array [nrhs], info dict).

    B: CUDA float64 [nrhs][N]; proj_idx: host int [nrhs][nproj] unit projections."""
    import torch
    n = scocg_dim(h)
    B = B if B.dim() == 2 else B.reshape(1, -1)
    _need(B.contiguous(), torch.float64, None, "B")
    B = B.contiguous()
    if B.shape[1] != n:
        raise ValueError("B rows must have the handle's dimension")
    nrhs = B.shape[0]
    pidx = np.ascontiguousarray(np.asarray(proj_idx, dtype=np.int64))
    if pidx.ndim == 1:
        pidx = np.ascontiguousarray(np.broadcast_to(pidx, (nrhs, pidx.size)))
    if pidx.shape[0] != nrhs:
        raise ValueError("proj_idx needs one row per right-hand side")
    M = pidx.shape[1]
    z, zp = _shifts(shifts)
    K = z.size
    G = torch.empty((nrhs, M, K), dtype=torch.complex128, device=B.device)
    used = np.zeros(nrhs, dtype=np.int32)
    sec = ctypes.c_double()
    code = lib().scocg_krylov_sd_multi(h.ptr, _dev(B), nrhs, int(nu), zp, K, pidx.ctypes.data, M, _dev(G),
                                       used.ctypes.data, ctypes.byref(sec))
    _check(code, "scocg_krylov_sd_multi")
    return G, used, {"status": code, "seconds": sec.value}


def scocg_krylov_sd(h: Handle, b, nu: int, shifts, proj_idx=None, proj_vec=None):
    """scocg_krylov_sd: returns (G [nproj][nshift] CUDA complex128, ritz [nu_used]
    CUDA float64, weight [nproj][nu_used] CUDA float64, info dict).

    b: CUDA float64 [N]; proj_idx: host int [nproj] or proj_vec: CUDA float64
    [nproj][N]."""
    import torch
    if b.dtype != torch.float64 or not b.is_cuda:
        raise TypeError("b must be a CUDA float64 tensor")
    n = scocg_dim(h)
    if b.numel() != n:
        raise ValueError("b must have the handle's dimension")
    b = b.reshape(-1).contiguous()
    z, zp = _shifts(shifts)
    K = z.size
    pidx_p = pvec_p = None
    keep = None
    if proj_idx is not None:
        keep = np.ascontiguousarray(np.asarray(proj_idx, dtype=np.int64).reshape(-1))
        M = keep.size
        pidx_p = keep.ctypes.data
    else:
        keep = (proj_vec if proj_vec.dim() == 2 else proj_vec.reshape(1, -1)).contiguous()
        if keep.dtype != torch.float64 or not keep.is_cuda:
            raise TypeError("proj_vec must be a CUDA float64 tensor")
        if keep.shape[1] != n:
            raise ValueError("proj_vec rows must have the handle's dimension")
        M = keep.shape[0]
        pvec_p = _dev(keep)
    G = torch.empty((M, K), dtype=torch.complex128, device=b.device)
    ritz = torch.zeros(int(nu), dtype=torch.float64, device=b.device)
    weight = torch.zeros((M, int(nu)), dtype=torch.float64, device=b.device)
    used = ctypes.c_int()
    sec = ctypes.c_double()
    code = lib().scocg_krylov_sd(h.ptr, _dev(b), int(nu), zp, K, pidx_p, pvec_p, M, _dev(G), _dev(ritz), _dev(weight),
                                 ctypes.byref(used), ctypes.byref(sec))
    _check(code, "scocg_krylov_sd")
    k = used.value
    return G, ritz[:k], weight[:, :k], {"status": code, "nu_used": k, "seconds": sec.value}


def scocg_excite(h_from: Handle, h_to: Handle, site: int, spin: int, create: bool, psi):
    """scocg_excite: c_{site,spin} psi (create=False) or c+_{site,spin} psi as a
    CUDA complex128 vector of h_to's sector."""
    import torch
    if psi.dtype != torch.float64 or not psi.is_cuda:
        raise TypeError("psi must be a CUDA float64 tensor")
    n = ctypes.c_int64()
    _check(lib().scocg_dim(h_to.ptr, ctypes.byref(n)), "scocg_dim")
    if psi.numel() != scocg_dim(h_from):
        raise ValueError("psi must have the source sector's dimension")
    out = torch.empty(n.value, dtype=torch.complex128, device=psi.device)
    psi = psi.reshape(-1).contiguous()
    _check(lib().scocg_excite(h_from.ptr, h_to.ptr, int(site), int(spin), int(bool(create)), _dev(psi), _dev(out)),
           "scocg_excite")
    return out


def scocg_hubbard_tables(h: Handle, spin: int):
    """Per-spin basis tables built on the device: (states, hop_target, hop_sign)."""
    d = ctypes.c_int32()
    _check(lib().scocg_hubbard_tables(h.ptr, spin, ctypes.byref(d), None, None, None), "scocg_hubbard_tables")
    D = d.value
    states = np.zeros(D, dtype=np.uint32)
    # slots per rank = 2L; recover L from the handle's dimension request below
    L2 = _hub_slots(h)
    tgt = np.zeros((D, L2), dtype=np.int32)
    sgn = np.zeros((D, L2), dtype=np.int8)
    _check(lib().scocg_hubbard_tables(h.ptr, spin, ctypes.byref(d), states.ctypes.data, tgt.ctypes.data,
                                      sgn.ctypes.data), "scocg_hubbard_tables")
    return states, tgt, sgn


def _hub_slots(h: Handle) -> int:
    return 2 * int(getattr(h, "L"))


def scocg_solve_csr_noalloc(rowptr32, col, val, shifts, rhs, proj_idx=None, proj_vec=None, tol: float = 1e-10,
                            max_iter: int = 0, G_out=None, stream=None):
    """scocg_solve_csr_noalloc: FP64 solve for callers that cannot allocate
    device memory; the library itself allocates nothing (its scratch is a fixed
    device array).  rowptr32/col: CUDA int32, val: CUDA float64, rhs: CUDA
    complex128 [N], proj_vec: CUDA complex128 [nproj][N] or proj_idx: host ints.
    G_out (CUDA complex128 [nproj][nshift]) may be passed in so that this call
    allocates nothing on the torch side either.  Returns (G, info)."""
    import torch
    z, zp = _shifts(shifts)
    K = z.size
    n = rowptr32.numel() - 1
    _need(rowptr32, torch.int32, None, "rowptr32")
    _need(col, torch.int32, None, "col")
    _need(val, torch.float64, col.numel(), "val")
    _need(rhs, torch.complex128, n, "rhs")
    pidx_p = pvec_p = None
    if proj_idx is not None:
        pidx = np.ascontiguousarray(np.asarray(proj_idx, dtype=np.int64).ravel())
        M = pidx.size
        pidx_p = pidx.ctypes.data
    else:
        M = proj_vec.shape[0] if proj_vec.dim() == 2 else 1
        _need(proj_vec, torch.complex128, M * n, "proj_vec")
        pvec_p = _dev(proj_vec)
    if G_out is None:
        G_out = torch.zeros((M, K), dtype=torch.complex128, device=rhs.device)
    _need(G_out, torch.complex128, M * K, "G_out")
    info, it, rs = _info_struct(1, K)
    code = lib().scocg_solve_csr_noalloc(n, col.numel(), _dev(rowptr32), _dev(col), _dev(val), zp, K, _dev(rhs),
                                         pidx_p, pvec_p, M, float(tol), int(max_iter), _dev(G_out),
                                         ctypes.byref(info), _stream_ptr(stream))
    _check(code, "scocg_solve_csr_noalloc")
    return G_out, _info_dict(info, it, rs, 1, K, code)


def scocg_solve_multi(handles, shifts, rhs, proj_idx=None, proj_vec=None, tol: float = 1e-10,
                      use_graph: bool = False, G_out=None):
    """scocg_solve_multi: independent systems in one launch.  handles, shifts,
    rhs (CUDA complex128 [N_s]) and proj_idx (host [nproj]) or proj_vec (CUDA
    complex128 [nproj][N_s]) are per-system lists.  Returns ([G_s], [info_s])."""
    import torch
    nsys = len(handles)
    hs = (ctypes.c_void_p * nsys)(*[h.ptr for h in handles])
    zs = [np.ascontiguousarray(np.asarray(z, dtype=np.complex128)) for z in shifts]
    zp = (ctypes.c_void_p * nsys)(*[z.ctypes.data for z in zs])
    ks = (ctypes.c_int * nsys)(*[z.size for z in zs])
    rhs = [r.reshape(-1).contiguous() for r in rhs]
    rp = (ctypes.c_void_p * nsys)(*[r.data_ptr() for r in rhs])
    keep = []
    if proj_idx is not None:
        pis = [np.ascontiguousarray(np.asarray(p, dtype=np.int64).ravel()) for p in proj_idx]
        keep.append(pis)
        pip = (ctypes.c_void_p * nsys)(*[p.ctypes.data for p in pis])
        pvp = None
        ms = [p.size for p in pis]
    else:
        pvs = [(p if p.dim() == 2 else p.reshape(1, -1)).contiguous() for p in proj_vec]
        keep.append(pvs)
        pvp = (ctypes.c_void_p * nsys)(*[p.data_ptr() for p in pvs])
        pip = None
        ms = [p.shape[0] for p in pvs]
    mp = (ctypes.c_int * nsys)(*ms)
    if G_out is None:
        G_out = [torch.zeros((m, z.size), dtype=torch.complex128, device=r.device) for m, z, r in zip(ms, zs, rhs)]
    gp = (ctypes.c_void_p * nsys)(*[g.data_ptr() for g in G_out])
    infos = (Info * nsys)()
    arrays = []
    for s in range(nsys):
        it = np.zeros(zs[s].size, dtype=np.int32)
        rs = np.zeros(zs[s].size, dtype=np.float64)
        infos[s].freeze_iter = it.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        infos[s].resid = rs.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        arrays.append((it, rs))
    code = lib().scocg_solve_multi(nsys, hs, zp, ks, rp, pip, pvp, mp, float(tol), gp, infos, int(bool(use_graph)))
    _check(code, "scocg_solve_multi")
    return G_out, [_info_dict(infos[s], arrays[s][0], arrays[s][1], 1, zs[s].size, code) for s in range(nsys)]


def scocg_multi_release() -> None:
    lib().scocg_multi_release()
