"""Seeded synthetic inputs shaped like the paper's workloads.

This module only synthesises inputs: tight-binding matrices in CSR form, shift
lists, right-hand sides and projection sets.  It contains none of the solver's
arithmetic, so the CUDA path and the CPU oracle can both be fed from it
without sharing any code that computes a result.

Workloads (the paper's own parameter sets are not available, so these stand in
for them with the same structure):

* ``chain``      -- one-orbital open chain with nearest-neighbour hopping t
                    (the textbook tight-binding form of Sec. II).
* ``anderson``   -- simple-cubic L^3 lattice with 4 orbitals per site, random
                    symmetric 4x4 onsite blocks U[-1,1] and random 4x4 hopping
                    blocks N(0, 0.25) on the 6 periodic neighbour bonds; every
                    entry is rounded to an FP32-representable double so that a
                    single-precision copy of H is exact.
* Hubbard ring parameters for the matrix-free extended Hubbard model of
  Sec. IV.B (the basis itself is built by each consumer).
* ``sqrt8_cluster`` and ``eg_model`` -- the doubly degenerate (two-orbital)
  extended Hubbard model on the sqrt(8) x sqrt(8) square-lattice cluster of
  Sec. IV.B, with synthetic hopping and interaction values (the paper's own
  parameter set is in a reference that is not available).

All randomness comes from numpy's PCG64 (``np.random.default_rng(seed)``).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "CSR", "chain_csr", "anderson_csr", "spectral_bounds", "random_unit_complex",
    "to_fp32_exact", "Workload", "workload", "cluster_sizes", "ANDERSON64_BOUNDS", "BATCH32_BOUNDS",
    "sqrt8_cluster", "eg_model",
]

# Spectral bounds (ARPACK, tol 1e-4) of the seed-2 64^3 x 4 Anderson matrix and
# of the seed-3 32^3 x 4 matrix, fixed so that every consumer draws the
# identical shift list without re-running the eigensolver.
ANDERSON64_BOUNDS = (-6.086151226927176, 6.469558282777935)
BATCH32_BOUNDS = (-6.041048698881869, 5.997536652116761)


@dataclass
class CSR:
    """Real symmetric sparse matrix in CSR form (rows sorted by column)."""
    n: int
    rowptr: np.ndarray  # int64 [n+1]
    col: np.ndarray     # int32 [nnz]
    val: np.ndarray     # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def dense(self) -> np.ndarray:
        return self.scipy().toarray()


def to_fp32_exact(a: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest FP32 value, kept as float64."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def _coo_to_csr(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate (row, col) entries")
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr, cols.astype(np.int32), vals.astype(np.float64))


def chain_csr(L: int, t: float = -1.0, onsite: float = 0.0) -> CSR:
    """Open chain of L sites, H_{i,i+1} = H_{i+1,i} = t; a zero onsite is not stored."""
    i = np.arange(L - 1, dtype=np.int64)
    rows = [i, i + 1]
    cols = [i + 1, i]
    vals = [np.full(L - 1, t), np.full(L - 1, t)]
    if onsite != 0.0:
        d = np.arange(L, dtype=np.int64)
        rows.append(d); cols.append(d); vals.append(np.full(L, onsite))
    return _coo_to_csr(L, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def anderson_csr(L: int, seed: int, norb: int = 4, hop_var: float = 0.25,
                 onsite_half_width: float = 1.0) -> CSR:
    """Periodic L^3 simple-cubic lattice, ``norb`` orbitals per site.

    Row index = norb * site + orbital, site = x + L*(y + L*z).  Onsite block:
    upper triangle drawn U[-w, w] and mirrored.  For every bond site -> site+d
    (d = +x, +y, +z, periodic) one norb x norb block M ~ N(0, hop_var) is drawn;
    block(site, site+d) = M and block(site+d, site) = M^T.  All values are
    rounded to FP32-representable doubles.  nnz = 7 * norb^2 per site.
    """
    if L < 3:
        raise ValueError("anderson_csr needs L >= 3 so that the 6 neighbours are distinct")
    rng = np.random.default_rng(seed)
    nsite = L ** 3
    n = nsite * norb
    site = np.arange(nsite, dtype=np.int64)
    x, y, z = site % L, (site // L) % L, site // (L * L)

    onsite = rng.uniform(-onsite_half_width, onsite_half_width, size=(nsite, norb, norb))
    iu = np.triu_indices(norb)
    sym = np.zeros_like(onsite)
    sym[:, iu[0], iu[1]] = onsite[:, iu[0], iu[1]]
    sym = sym + np.transpose(sym, (0, 2, 1))
    sym[:, np.arange(norb), np.arange(norb)] *= 0.5

    std = math.sqrt(hop_var)
    hops = rng.normal(0.0, std, size=(3, nsite, norb, norb))
    nb = [
        ((x + 1) % L) + L * (y + L * z),
        x + L * (((y + 1) % L) + L * z),
        x + L * (y + L * ((z + 1) % L)),
    ]

    oi, oj = np.meshgrid(np.arange(norb), np.arange(norb), indexing="ij")
    oi = oi.ravel(); oj = oj.ravel()
    rows, cols, vals = [], [], []

    def add_block(src_site, dst_site, blocks):
        rows.append((norb * src_site[:, None] + oi[None, :]).ravel())
        cols.append((norb * dst_site[:, None] + oj[None, :]).ravel())
        vals.append(blocks.reshape(len(src_site), -1).ravel())

    add_block(site, site, sym)
    for d in range(3):
        add_block(site, nb[d], hops[d])
        add_block(nb[d], site, np.transpose(hops[d], (0, 2, 1)))
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    vals = to_fp32_exact(np.concatenate(vals))
    return _coo_to_csr(n, rows, cols, vals)


def spectral_bounds(h: CSR, tol: float = 1e-4) -> tuple[float, float]:
    """Lowest and highest eigenvalue of H from ARPACK (scipy.sparse.linalg.eigsh)."""
    from scipy.sparse.linalg import eigsh
    a = h.scipy()
    v0 = np.ones(h.n) / math.sqrt(h.n)
    hi = eigsh(a, k=1, which="LA", tol=tol, v0=v0, return_eigenvectors=False)[0]
    lo = eigsh(a, k=1, which="SA", tol=tol, v0=v0, return_eigenvectors=False)[0]
    return float(lo), float(hi)


def random_unit_complex(n: int, seed: int) -> np.ndarray:
    """Seeded complex vector with N(0,1) real and imaginary parts, normalised to 1."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=n) + 1j * rng.normal(size=n)
    return v / np.linalg.norm(v)


def random_unit_real(n: int, seed: int) -> np.ndarray:
    """Seeded real vector with N(0,1) entries, normalised to 1 (a start vector)."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=n)
    return v / np.linalg.norm(v)


def cluster_sizes(nsys: int = 32, lmin: int = 14, lmax: int = 50, seed: int = 31) -> np.ndarray:
    """Edge lengths of the uneven Anderson clusters of the multi-system batch."""
    rng = np.random.default_rng(seed)
    return rng.integers(lmin, lmax + 1, size=nsys)


def sqrt8_cluster() -> tuple[list[tuple[int, int]], list[int]]:
    """The 8-site sqrt(8) x sqrt(8) cluster of the square lattice with periodic
    boundary conditions: lattice points (x, y) modulo the vectors (2, 2) and
    (2, -2), represented by 0 <= x < 4, 0 <= y < 2 (site = x + 4 y).  Returns
    the 16 nearest-neighbour bonds (i, j) (each site to its +x and +y
    neighbour) and the direction of each bond (0 = x, 1 = y)."""
    def site(x, y):
        while y >= 2:
            x, y = x - 2, y - 2
        while y < 0:
            x, y = x + 2, y + 2
        return (x % 4) + 4 * y
    bonds, dirs = [], []
    for y in range(2):
        for x in range(4):
            for d, (dx, dy) in enumerate(((1, 0), (0, 1))):
                bonds.append((site(x, y), site(x + dx, y + dy)))
                dirs.append(d)
    return bonds, dirs


# Synthetic values standing in for the two-orbital model's parameters: e_g-like
# hoppings (orbital 0 ~ x^2-y^2, orbital 1 ~ 3z^2-r^2) whose inter-orbital
# element changes sign between the x and y bonds, Kanamori on-site terms with
# U' = U - 2 J and J' = J, and the inter-site Coulomb V.  Every value is a
# dyadic rational, so H has the same entries in FP64 and FP32.
EG_HOPPING = {0: ((-0.75, 0.4375), (0.4375, -0.25)), 1: ((-0.75, -0.4375), (-0.4375, -0.25))}
EG_INTERACTION = {"U": 4.0, "Up": 2.5, "J": 0.75, "Jp": 0.75, "V": 1.0}


def eg_model(bonds=None, dirs=None, **over) -> dict:
    """The two-orbital extended Hubbard model on a bond list (default: the
    sqrt(8) x sqrt(8) cluster) with the synthetic values above; keyword
    arguments override U, Up, J, Jp, V."""
    if bonds is None:
        bonds, dirs = sqrt8_cluster()
    n_sites = 1 + max(max(b) for b in bonds)
    bond_t = [list(map(list, EG_HOPPING[d])) for d in dirs]
    m = {"n_sites": n_sites, "bonds": [tuple(b) for b in bonds], "dirs": list(dirs), "bond_t": bond_t}
    m.update(EG_INTERACTION)
    m.update(over)
    return m


@dataclass
class Workload:
    """One synthetic problem: H (CSR or Hubbard parameters), shifts, rhs, projections."""
    name: str
    shifts: np.ndarray                       # complex128 [nshift]
    rhs: np.ndarray                          # complex128 [nrhs][n]
    tol: float
    csr: CSR | None = None
    hubbard: dict | None = None
    proj_idx: np.ndarray | None = None       # int64 [nrhs][nproj]
    proj_vec: np.ndarray | None = None       # complex128 [nproj][n]
    weights: np.ndarray | None = None        # float64 [nshift] (spectral loss)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.csr.n if self.csr is not None else int(self.rhs.shape[1])


def _unit(n: int, j: int) -> np.ndarray:
    e = np.zeros(n, dtype=np.complex128)
    e[j] = 1.0
    return e


def workload(name: str, scale: str = "full", bounds: tuple[float, float] | None = None) -> Workload:
    """Synthetic workloads.

    name:
      ``chain``     open chain L=4096 (scale "small": L=256), t=-1, b=e_0,
                    64 shifts linspace(-2.5, 2.5) + 0.01i, tol 1e-10.
      ``anderson``  64^3 x 4 Anderson (scale "small": 6^3 x 4, "medium": 16^3 x 4),
                    b seeded unit complex, c = conj(b), 512 shifts seeded-uniform
                    over [lambda_min, lambda_max] + 1e-3 i, tol 1e-6.
      ``batch``     32^3 x 4 Anderson (small: 6^3 x 4), 256 rhs e_j at distinct
                    seeded rows with projection e_j, 256 shifts evenly over the
                    bounds + 1e-2 i (small: 32 rhs, 32 shifts).
      ``adjoint``   24^3 x 4 Anderson (small: 4^3 x 4), b = c = e_0, 128 shifts
                    evenly over the bounds + 0.02 i, weights N(0,1).
      ``hubbard``   L=14 ring, 7 up 7 down, t=1, U=4, V=1, periodic; b seeded unit
                    complex, c = conj(b), 128 shifts linspace(-10, 20) + 0.05i
                    (small: L=8, 4 up 4 down).
      ``hubbard2``  two-orbital extended Hubbard model on the sqrt(8) x sqrt(8)
                    cluster, 6 up 6 down (64,128,064 states; medium 3/3:
                    313,600; small 2/2: 14,400), eg_model values, b seeded unit
                    complex, c = conj(b), 128 shifts linspace(-12, 48) + 0.1i.
    """
    if name == "chain":
        L = 4096 if scale == "full" else 256
        h = chain_csr(L, t=-1.0)
        shifts = np.linspace(-2.5, 2.5, 64) + 0.01j
        return Workload(name, shifts, _unit(L, 0)[None, :], 1e-10, csr=h,
                        proj_idx=np.zeros((1, 1), dtype=np.int64), meta={"L": L, "seed": 1})
    if name == "anderson":
        L = {"full": 64, "medium": 16, "small": 6}[scale]
        h = anderson_csr(L, seed=2)
        lo, hi = bounds if bounds is not None else spectral_bounds(h)
        rng = np.random.default_rng(2)
        e = np.sort(rng.uniform(lo, hi, 512))
        b = random_unit_complex(h.n, seed=2)
        return Workload(name, e + 1e-3j, b[None, :], 1e-6, csr=h,
                        proj_vec=np.conj(b)[None, :], meta={"L": L, "seed": 2, "bounds": (lo, hi)})
    if name == "batch":
        L, nrhs, nshift = {"full": (32, 256, 256), "small": (6, 32, 32)}[scale]
        h = anderson_csr(L, seed=3)
        lo, hi = bounds if bounds is not None else spectral_bounds(h)
        rng = np.random.default_rng(3)
        sites = rng.choice(h.n, size=nrhs, replace=False).astype(np.int64)
        rhs = np.zeros((nrhs, h.n), dtype=np.complex128)
        rhs[np.arange(nrhs), sites] = 1.0
        shifts = np.linspace(lo, hi, nshift) + 1e-2j
        return Workload(name, shifts, rhs, 1e-6, csr=h, proj_idx=sites[:, None].copy(),
                        meta={"L": L, "seed": 3, "bounds": (lo, hi)})
    if name == "adjoint":
        L = {"full": 24, "small": 4}[scale]
        h = anderson_csr(L, seed=4)
        lo, hi = bounds if bounds is not None else spectral_bounds(h)
        rng = np.random.default_rng(4)
        shifts = np.linspace(lo, hi, 128) + 0.02j
        w = rng.normal(size=128)
        return Workload(name, shifts, _unit(h.n, 0)[None, :], 1e-10, csr=h,
                        proj_idx=np.zeros((1, 1), dtype=np.int64), weights=w,
                        meta={"L": L, "seed": 4, "bounds": (lo, hi)})
    if name == "hubbard":
        L, nup = {"full": (14, 7), "small": (8, 4)}[scale]
        n = math.comb(L, nup) ** 2
        b = random_unit_complex(n, seed=5)
        shifts = np.linspace(-10.0, 20.0, 128) + 0.05j
        hub = dict(L=L, n_up=nup, n_dn=nup, t=1.0, U=4.0, V=1.0, periodic=True)
        return Workload(name, shifts, b[None, :], 1e-6, hubbard=hub,
                        proj_vec=np.conj(b)[None, :], meta={"seed": 5, **hub})
    if name == "hubbard2":
        n_el = {"full": 6, "medium": 3, "small": 2}[scale]
        model = eg_model()
        n = math.comb(16, n_el) ** 2
        b = random_unit_complex(n, seed=6)
        shifts = np.linspace(-12.0, 48.0, 128) + 0.1j
        return Workload(name, shifts, b[None, :], 1e-8, hubbard=model, proj_vec=np.conj(b)[None, :],
                        meta={"seed": 6, "n_up": n_el, "n_dn": n_el})
    raise ValueError(f"unknown workload {name!r}")
