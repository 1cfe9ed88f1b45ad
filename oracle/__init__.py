"""CPU oracle for the shifted-COCG Green's-function solver.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product path never imports it and
shares no code with it (the seeded inputs come from a separate module that does
no solver arithmetic).

Contents (each function cites the passage of arXiv:0802.0748 it follows):

* ``shifted_cocg``       plain FP64 C shifted COCG with full per-shift vectors
                         and seed switching (Sec. III.C; Eqs. lin_eq,
                         shift_lin_eq, residual).
* ``apply_shifted``      y = (z I - H) x (Eq. lin_eq's matrix).
* ``hubbard_csr``        extended Hubbard sector Hamiltonian from the literal
                         Jordan-Wigner definition (Sec. IV.B).
* ``hubbard2_csr``,      the two-orbital (doubly degenerate) extended Hubbard
  ``hubbard2_rows``      model of Sec. IV.B: sector CSR, or sampled rows of H x
                         for sectors too large for CSR.
* ``grad_from_vectors``  dL/dH on the stored entries from the full solutions of
                         the forward and adjoint shifted systems.
* ``dense``              dense LU Green's functions, closed forms, Fock-space
                         exact diagonalisation, dense gradients.
* ``ground``             Lanczos / CG-inverse-iteration ground state and the
                         one-particle operators c, c+ between sectors
                         (Sec. II.B, Sec. IV.B).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
LIB_PATH = HERE / "_build" / "liboracle.so"
SRC = HERE / "scocg_oracle.c"

OK, NOT_CONVERGED, ERR_INVALID, ERR_OOM, ERR_BREAKDOWN = 0, 1, -1, -3, -4


def build(force: bool = False) -> Path:
    """Compile the C oracle with gcc (OpenMP) into oracle/_build/liboracle.so."""
    LIB_PATH.parent.mkdir(exist_ok=True)
    if force or not LIB_PATH.exists() or LIB_PATH.stat().st_mtime < SRC.stat().st_mtime:
        tmp = LIB_PATH.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-o", str(tmp), str(SRC), "-lm"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(LIB_PATH))
        P = ctypes.c_void_p
        L.oracle_shifted_cocg.restype = ctypes.c_int
        L.oracle_shifted_cocg.argtypes = [
            ctypes.c_int64, P, P, P, ctypes.c_int, P, P, ctypes.c_int, P, P,
            ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
            P, P, P, P, P, P, P]
        L.oracle_apply_shifted.restype = None
        L.oracle_apply_shifted.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_double,
                                           ctypes.c_double, P, P]
        L.oracle_hubbard_csr.restype = ctypes.c_int64
        L.oracle_hubbard_csr.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [ctypes.c_int, P, P, P]
        L.oracle_sector_dim.restype = ctypes.c_int64
        L.oracle_sector_dim.argtypes = [ctypes.c_int, ctypes.c_int]
        L.oracle_default_seed.restype = ctypes.c_int
        L.oracle_default_seed.argtypes = [ctypes.c_int, P]
        h2 = [ctypes.c_int, ctypes.c_int, P, P, P] + [ctypes.c_double] * 5 + [ctypes.c_int, ctypes.c_int]
        L.oracle_hubbard2_csr.restype = ctypes.c_int64
        L.oracle_hubbard2_csr.argtypes = h2 + [P, P, P]
        L.oracle_hubbard2_rows.restype = ctypes.c_int
        L.oracle_hubbard2_rows.argtypes = h2 + [ctypes.c_int64, P, P, P]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _csr_arrays(rowptr, col, val):
    return (np.ascontiguousarray(rowptr, dtype=np.int64), np.ascontiguousarray(col, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))


class Result:
    """Output of one oracle solve."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def shifted_cocg(rowptr, col, val, shifts, b, *, proj_idx=None, proj_vec=None, tol=1e-10,
                 max_iter=100000, seed=-1, allow_switch=True, want_x=False, want_state=False) -> Result:
    """Shifted COCG (Sec. III.C) for one right-hand side ``b`` and all ``shifts``.

    Returns G[nproj][nshift] (G_mk = c_m^T x^k, Eq. gf), per-shift iteration
    counts and residuals ||r^k||/||b||, the status code, statistics (iterations,
    shift-iterations, switches, final seed) and optionally the full solutions
    X[nshift][n] and the final seed residual / pi^k.
    """
    rowptr, col, val = _csr_arrays(rowptr, col, val)
    n = rowptr.size - 1
    z = np.ascontiguousarray(shifts, dtype=np.complex128)
    bb = np.ascontiguousarray(b, dtype=np.complex128)
    if bb.shape != (n,):
        raise ValueError("b must have shape (n,)")
    K = z.size
    pidx = None if proj_idx is None else np.ascontiguousarray(proj_idx, dtype=np.int64).ravel()
    pvec = None if proj_vec is None else np.ascontiguousarray(proj_vec, dtype=np.complex128).reshape(-1, n)
    nproj = pidx.size if pidx is not None else (pvec.shape[0] if pvec is not None else 0)
    G = np.zeros((max(nproj, 1), K), dtype=np.complex128)
    iters = np.zeros(K, dtype=np.int32)
    resid = np.zeros(K, dtype=np.float64)
    X = np.zeros((K, n), dtype=np.complex128) if want_x else None
    r_out = np.zeros(n, dtype=np.complex128) if want_state else None
    pi_out = np.zeros(K, dtype=np.complex128) if want_state else None
    stats = np.zeros(4, dtype=np.float64)
    st = lib().oracle_shifted_cocg(n, _ptr(rowptr), _ptr(col), _ptr(val), K, _ptr(z), _ptr(bb),
                                   nproj, _ptr(pidx), _ptr(pvec), float(tol), int(max_iter),
                                   int(seed), int(bool(allow_switch)), _ptr(G), _ptr(iters),
                                   _ptr(resid), _ptr(X), _ptr(r_out), _ptr(pi_out), _ptr(stats))
    return Result(status=st, G=G[:nproj], iters=iters, resid=resid, X=X, r=r_out, pi=pi_out,
                  n_iter=int(stats[0]), shift_iters=int(stats[1]), n_switch=int(stats[2]),
                  seed=int(stats[3]))


def default_seed(shifts) -> int:
    """Seed rule: smallest Im z, then Re z nearest the median, then lowest index."""
    z = np.ascontiguousarray(shifts, dtype=np.complex128)
    return int(lib().oracle_default_seed(z.size, _ptr(z)))


def apply_shifted(rowptr, col, val, z: complex, x) -> np.ndarray:
    """y = (z I - H) x with H in CSR (Eq. lin_eq's matrix)."""
    rowptr, col, val = _csr_arrays(rowptr, col, val)
    xx = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.empty_like(xx)
    lib().oracle_apply_shifted(rowptr.size - 1, _ptr(rowptr), _ptr(col), _ptr(val),
                               float(np.real(z)), float(np.imag(z)), _ptr(xx), _ptr(y))
    return y


def sector_dim(L: int, k: int) -> int:
    """Number of L-bit strings with k ones, counted by enumeration (Sec. IV.B)."""
    return int(lib().oracle_sector_dim(L, k))


def hubbard_csr(L, n_up, n_dn, t, U, V, periodic=True):
    """Extended Hubbard sector Hamiltonian in CSR from the literal Jordan-Wigner
    definition (Sec. IV.B).  Returns (rowptr, col, val)."""
    f = lib().oracle_hubbard_csr
    nnz = f(L, n_up, n_dn, t, U, V, int(periodic), None, None, None)
    if nnz < 0:
        raise ValueError(f"hubbard_csr failed ({nnz})")
    dim = sector_dim(L, n_up) * sector_dim(L, n_dn)
    rowptr = np.zeros(dim + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz, dtype=np.float64)
    nnz2 = f(L, n_up, n_dn, t, U, V, int(periodic), _ptr(rowptr), _ptr(col), _ptr(val))
    assert nnz2 == nnz
    return rowptr, col, val


def grad_from_vectors(rowptr, col, X, Y, gbar) -> np.ndarray:
    """Gradient of a real loss L(G) with respect to every stored value of H.

    G_k = c^T (z_k I - H)^{-1} b (Eq. gf with a projection c), so with
    x_k = (z_k I - H)^{-1} b and y_k = (z_k I - H)^{-T} c (the same matrix: it is
    complex symmetric, Sec. III.C) the derivative by one stored entry (a, b)
    treated as an independent parameter is dG_k/dH_ab = y_k[a] x_k[b]; for
    gbar_k = dL/dRe G_k + i dL/dIm G_k, dL/dH_ab = Re sum_k conj(gbar_k)
    y_k[a] x_k[b].  X, Y: [nshift][n] complex; returns float64 [nnz] in CSR order.
    """
    rowptr = np.asarray(rowptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    X = np.asarray(X, dtype=np.complex128)
    Y = np.asarray(Y, dtype=np.complex128)
    w = np.conj(np.asarray(gbar, dtype=np.complex128))
    rows = np.repeat(np.arange(rowptr.size - 1, dtype=np.int64), np.diff(rowptr))
    g = np.zeros(col.size, dtype=np.float64)
    step = 1 << 16
    for e0 in range(0, col.size, step):            # sum over k for a block of entries
        a = rows[e0:e0 + step]
        bcol = col[e0:e0 + step]
        g[e0:e0 + step] = np.real(np.einsum("k,ke,ke->e", w, Y[:, a], X[:, bcol]))
    return g


def _model2_args(model):
    bi = np.ascontiguousarray([b[0] for b in model["bonds"]], dtype=np.int32)
    bj = np.ascontiguousarray([b[1] for b in model["bonds"]], dtype=np.int32)
    bt = np.ascontiguousarray(model["bond_t"], dtype=np.float64).reshape(-1, 2, 2)
    if bt.shape[0] != bi.size:
        raise ValueError("bond_t must hold one 2x2 block per bond")
    keep = (bi, bj, bt)
    args = [int(model["n_sites"]), int(bi.size), _ptr(bi), _ptr(bj), _ptr(bt), float(model["U"]),
            float(model["Up"]), float(model["J"]), float(model["Jp"]), float(model["V"])]
    return args, keep


def hubbard2_csr(model, n_up, n_dn):
    """Two-orbital extended Hubbard sector Hamiltonian (Sec. IV.B) in CSR, built
    from the literal Jordan-Wigner definition of every term.  ``model``: dict
    with n_sites, bonds [(i, j)], bond_t [nb][2][2], U, Up, J, Jp, V.
    Returns (rowptr, col, val)."""
    args, keep = _model2_args(model)
    f = lib().oracle_hubbard2_csr
    nnz = f(*args, int(n_up), int(n_dn), None, None, None)
    if nnz < 0:
        raise ValueError(f"hubbard2_csr failed ({nnz})")
    M = 2 * int(model["n_sites"])
    dim = math.comb(M, n_up) * math.comb(M, n_dn)
    rowptr = np.zeros(dim + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz, dtype=np.float64)
    nnz2 = f(*args, int(n_up), int(n_dn), _ptr(rowptr), _ptr(col), _ptr(val))
    assert nnz2 == nnz
    return rowptr, col, val


def hubbard2_rows(model, n_up, n_dn, rows, x) -> np.ndarray:
    """(H x)[rows] of the two-orbital model's sector, each row from the terms of
    H applied to its basis state (for sectors too large for CSR)."""
    args, keep = _model2_args(model)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    xx = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.zeros(r.size, dtype=np.complex128)
    st = lib().oracle_hubbard2_rows(*args, int(n_up), int(n_dn), r.size, _ptr(r), _ptr(xx), _ptr(y))
    if st != 0:
        raise ValueError(f"hubbard2_rows failed ({st})")
    return y
