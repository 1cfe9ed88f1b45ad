"""Dense and closed-form references (TEST INFRASTRUCTURE ONLY).

Each function is the plain definition it names, with a library routine
(LAPACK through numpy) as its only step:

* ``green_dense``     G_mk = c_m^T (z_k I - H)^{-1} b by dense LU (Eq. gf / lin_eq).
* ``chain_g00_*``     Green's function of the one-orbital open chain: the exact
                      finite-chain eigen-sum, the semi-infinite surface form and
                      the bulk form (textbook tight-binding results for the
                      chain Hamiltonian of Sec. II).
* ``fock_hubbard``    extended Hubbard Hamiltonian of Sec. IV.B built in the full
                      4^L Fock space from Jordan-Wigner Kronecker products, then
                      restricted to an (N_up, N_dn) sector.
* ``fock_hubbard2``   the two-orbital extended Hubbard model of Sec. IV.B
                      (Kanamori on-site interaction) in the full Fock space of
                      a small cluster, plus its spin operators.
* ``grad_dense``      dG/dH_ab = (A^{-T} c)_a (A^{-1} b)_b from the dense inverse.
* ``fermi``, ``density_exact``, ``density_quadrature``  the density matrix of
                      Eqs. densityM-1 / densityM: the Fermi-weighted eigenstate
                      sum (dense eigendecomposition) and the real-axis Fermi
                      integral of given Green's functions on a uniform grid.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def green_dense(H: np.ndarray, shifts, b, C) -> np.ndarray:
    """G[m, k] = C[m]^T (z_k I - H)^{-1} b by dense LU (Eq. gf, Eq. lin_eq)."""
    n = H.shape[0]
    C = np.atleast_2d(np.asarray(C, dtype=np.complex128))
    out = np.empty((C.shape[0], len(shifts)), dtype=np.complex128)
    for k, z in enumerate(shifts):
        x = np.linalg.solve(z * np.eye(n) - H, b)
        out[:, k] = C @ x
    return out


def chain_g00_exact(L: int, t: float, z) -> np.ndarray:
    """Site-0 Green's function of an open chain of L sites with hopping t:
    eigenvectors sqrt(2/(L+1)) sin(n pi j/(L+1)), eigenvalues 2 t cos(n pi/(L+1))."""
    z = np.asarray(z, dtype=np.complex128)
    m = np.arange(1, L + 1)
    th = m * np.pi / (L + 1)
    w = (2.0 / (L + 1)) * np.sin(th) ** 2
    e = 2.0 * t * np.cos(th)
    return (w[None, :] / (z.reshape(-1, 1) - e[None, :])).sum(axis=1)


def chain_g00_surface(t: float, z) -> np.ndarray:
    """Semi-infinite chain, end site: g = (z - sqrt(z - 2|t|) sqrt(z + 2|t|)) / (2 t^2)."""
    z = np.asarray(z, dtype=np.complex128)
    a = 2.0 * abs(t)
    return (z - np.sqrt(z - a) * np.sqrt(z + a)) / (2.0 * t * t)


def chain_gjj_bulk(t: float, z) -> np.ndarray:
    """Infinite chain, any site: G = 1 / (sqrt(z - 2|t|) sqrt(z + 2|t|)) (= 1/sqrt(z^2 - 4t^2))."""
    z = np.asarray(z, dtype=np.complex128)
    a = 2.0 * abs(t)
    return 1.0 / (np.sqrt(z - a) * np.sqrt(z + a))


# --------------------------------------------------------------------------
# Fock-space construction (independent of any bit-string ranking scheme)
# --------------------------------------------------------------------------

def _jw_annihilators(nmodes: int):
    """c_m = Z x ... x Z x a x 1 x ... x 1 (Jordan-Wigner), mode 0 leftmost.

    Basis index of an occupation pattern (n_0, ..., n_{M-1}) is sum n_m 2^(M-1-m),
    i.e. mode 0 is the most significant bit of the Kronecker index."""
    a = np.array([[0.0, 1.0], [0.0, 0.0]])   # |0><1| in basis (|0>, |1>)
    Z = np.diag([1.0, -1.0])
    I2 = np.eye(2)
    ops = []
    for m in range(nmodes):
        mats = [Z] * m + [a] + [I2] * (nmodes - m - 1)
        op = mats[0]
        for x in mats[1:]:
            op = np.kron(op, x)
        ops.append(op)
    return ops


def hubbard_bonds(L: int, periodic: bool):
    bonds = [(i, i + 1) for i in range(L - 1)]
    if periodic and L >= 3:
        bonds.append((L - 1, 0))
    return bonds


def fock_hubbard(L: int, t: float, U: float, V: float, periodic: bool = True):
    """Extended Hubbard Hamiltonian (Sec. IV.B) on the full 4^L Fock space.

    H = -t sum_{<ij>,s} (c+_is c_js + h.c.) + U sum_i n_iu n_id + V sum_<ij> n_i n_j.
    Modes: up-spin sites 0..L-1 are modes 0..L-1, down-spin sites are modes L..2L-1.
    Returns (H, occupations) where occupations[idx] is the tuple of 2L mode
    occupations of Kronecker basis state idx."""
    M = 2 * L
    c = _jw_annihilators(M)
    cd = [x.T for x in c]
    num = [cd[m] @ c[m] for m in range(M)]
    H = np.zeros((2 ** M, 2 ** M))
    for (i, j) in hubbard_bonds(L, periodic):
        for s in range(2):
            a, b = i + s * L, j + s * L
            H += -t * (cd[a] @ c[b] + cd[b] @ c[a])
        ni = num[i] + num[i + L]
        nj = num[j] + num[j + L]
        H += V * ni @ nj
    for i in range(L):
        H += U * num[i] @ num[i + L]
    occ = [tuple((idx >> (M - 1 - m)) & 1 for m in range(M)) for idx in range(2 ** M)]
    return H, occ


def sector_states(L: int, k: int):
    """Bit strings (bit i = site i) with k ones, in ascending numeric order."""
    return [s for s in range(1 << L) if bin(s).count("1") == k]


def fock_hubbard_sector(L, n_up, n_dn, t, U, V, periodic=True) -> np.ndarray:
    """Sector block of ``fock_hubbard`` in the basis index rank_up * D_dn + rank_dn,
    rank = position among same-popcount strings in ascending order."""
    H, occ = fock_hubbard(L, t, U, V, periodic)
    ups, dns = sector_states(L, n_up), sector_states(L, n_dn)
    M = 2 * L
    idx = []
    for u in ups:
        for d in dns:
            bits = [(u >> i) & 1 for i in range(L)] + [(d >> i) & 1 for i in range(L)]
            idx.append(sum(bits[m] << (M - 1 - m) for m in range(M)))
    idx = np.array(idx)
    return H[np.ix_(idx, idx)]


def free_fermion_sector_spectrum(L: int, n_up: int, n_dn: int, t: float) -> np.ndarray:
    """All many-body energies of -t sum (c+_i c_{i+1} + h.c.) on a periodic ring:
    sums over occupied momenta of -2 t cos(2 pi m / L), for each spin."""
    eps = -2.0 * t * np.cos(2 * np.pi * np.arange(L) / L)
    up = [sum(eps[list(c)]) for c in itertools.combinations(range(L), n_up)]
    dn = [sum(eps[list(c)]) for c in itertools.combinations(range(L), n_dn)]
    return np.sort(np.add.outer(np.array(up), np.array(dn)).ravel())


def two_site_spectrum(t: float, U: float, V: float) -> np.ndarray:
    """Two sites, one bond, one up and one down electron: {V, U, (U+V)/2 +- sqrt(((U-V)/2)^2 + 4t^2)}."""
    s = math.sqrt(((U - V) / 2) ** 2 + 4 * t * t)
    return np.sort(np.array([V, U, (U + V) / 2 - s, (U + V) / 2 + s]))


def fock_hubbard2(model):
    """Two-orbital extended Hubbard Hamiltonian (Sec. IV.B) on the full Fock
    space of 4 ns modes from Jordan-Wigner Kronecker products:

      H = sum_bonds sum_ab sum_s t_ab (c+_ias c_jbs + h.c.) + U sum_ia n_ia,up n_ia,dn
        + U' sum_i n_i0 n_i1 - J sum_is n_i0s n_i1s
        + J sum_is c+_i0s c+_i1s' c_i0s' c_i1s + J' sum_i (c+_i0u c+_i0d c_i1d c_i1u + h.c.)
        + V sum_bonds n_i n_j.

    Modes: spin s, site i, orbital a -> 2 i + a + s 2 ns (mode 0 is the most
    significant bit of the Kronecker index).  Returns (H, c, M) with c the list
    of annihilators."""
    ns = int(model["n_sites"])
    M = 4 * ns
    c = _jw_annihilators(M)
    cd = [x.T for x in c]
    num = [cd[m] @ c[m] for m in range(M)]
    mode = lambda i, a, s: 2 * i + a + s * 2 * ns
    H = np.zeros((2 ** M, 2 ** M))
    for (i, j), t in zip(model["bonds"], np.asarray(model["bond_t"], dtype=np.float64).reshape(-1, 2, 2)):
        for a in range(2):
            for b in range(2):
                for s in range(2):
                    H += t[a, b] * (cd[mode(i, a, s)] @ c[mode(j, b, s)] + cd[mode(j, b, s)] @ c[mode(i, a, s)])
        ni = sum(num[mode(i, a, s)] for a in range(2) for s in range(2))
        nj = sum(num[mode(j, a, s)] for a in range(2) for s in range(2))
        H += model["V"] * ni @ nj
    for i in range(ns):
        for a in range(2):
            H += model["U"] * num[mode(i, a, 0)] @ num[mode(i, a, 1)]
        n0 = num[mode(i, 0, 0)] + num[mode(i, 0, 1)]
        n1 = num[mode(i, 1, 0)] + num[mode(i, 1, 1)]
        H += model["Up"] * n0 @ n1
        for s in range(2):
            so = 1 - s
            H -= model["J"] * num[mode(i, 0, s)] @ num[mode(i, 1, s)]
            H += model["J"] * cd[mode(i, 0, s)] @ cd[mode(i, 1, so)] @ c[mode(i, 0, so)] @ c[mode(i, 1, s)]
        P = cd[mode(i, 0, 0)] @ cd[mode(i, 0, 1)] @ c[mode(i, 1, 1)] @ c[mode(i, 1, 0)]
        H += model["Jp"] * (P + P.T)
    return H, c, M


def fock_spin2(ns: int, c):
    """Total S^2 and S_z of the two-orbital cluster (modes as in fock_hubbard2)."""
    M = 4 * ns
    cd = [x.T for x in c]
    up = [2 * i + a for i in range(ns) for a in range(2)]
    dn = [m + 2 * ns for m in up]
    Sp = sum(cd[u] @ c[d] for u, d in zip(up, dn))
    Sz = 0.5 * sum(cd[u] @ c[u] - cd[d] @ c[d] for u, d in zip(up, dn))
    S2 = Sp.T @ Sp + Sz @ Sz + Sz
    return S2, Sz


def fock_sector2(H: np.ndarray, ns: int, n_up: int, n_dn: int) -> np.ndarray:
    """Sector block of a two-orbital Fock-space operator in the basis index
    rank_up * D_dn + rank_dn (per-spin strings of 2 ns bits, bit m = mode m,
    ranked among same-popcount strings in ascending order)."""
    L = 2 * ns
    M = 2 * L
    ups, dns = sector_states(L, n_up), sector_states(L, n_dn)
    idx = []
    for u in ups:
        for d in dns:
            bits = [(u >> i) & 1 for i in range(L)] + [(d >> i) & 1 for i in range(L)]
            idx.append(sum(bits[m] << (M - 1 - m) for m in range(M)))
    idx = np.array(idx)
    return H[np.ix_(idx, idx)]


def kanamori_two_electron_levels(U: float, Up: float, J: float, Jp: float) -> np.ndarray:
    """One site, two orbitals, one up and one down electron: the four levels
    U' - J (S_z = 0 partner of the triplet), U' + J, U - J', U + J'."""
    return np.sort(np.array([Up - J, Up + J, U - Jp, U + Jp]))


def hopping_matrix2(model) -> np.ndarray:
    """Single-particle hopping matrix of one spin (index 2 i + a)."""
    ns = int(model["n_sites"])
    T = np.zeros((2 * ns, 2 * ns))
    for (i, j), t in zip(model["bonds"], np.asarray(model["bond_t"], dtype=np.float64).reshape(-1, 2, 2)):
        for a in range(2):
            for b in range(2):
                T[2 * i + a, 2 * j + b] += t[a, b]
                T[2 * j + b, 2 * i + a] += t[a, b]
    return T


def free_fermion_spectrum2(model, n_up: int, n_dn: int) -> np.ndarray:
    """All energies of the hopping part alone in a sector: sums of occupied
    eigenvalues of the single-particle hopping matrix, for each spin."""
    eps = np.linalg.eigvalsh(hopping_matrix2(model))
    up = [sum(eps[list(c)]) for c in itertools.combinations(range(eps.size), n_up)]
    dn = [sum(eps[list(c)]) for c in itertools.combinations(range(eps.size), n_dn)]
    return np.sort(np.add.outer(np.array(up), np.array(dn)).ravel())


def grad_dense(H: np.ndarray, shifts, b, c, gbar) -> np.ndarray:
    """dL/dH_ab for L real with dL/dG_k = gbar_k (torch convention dL/dRe + i dL/dIm):
    g_ab = Re sum_k conj(gbar_k) (A_k^{-T} c)_a (A_k^{-1} b)_b, A_k = z_k I - H."""
    n = H.shape[0]
    g = np.zeros((n, n))
    for k, z in enumerate(shifts):
        A = z * np.eye(n) - H
        x = np.linalg.solve(A, b)
        y = np.linalg.solve(A.T, c)
        g += np.real(np.conj(gbar[k]) * np.outer(y, x))
    return g


def fermi(e, mu: float, kT: float):
    """Fermi-Dirac occupation f((e - mu)/kT) of Eq. densityM; kT = 0 is the
    step function (1/2 at e = mu)."""
    e = np.asarray(e, dtype=np.float64)
    if kT <= 0.0:
        return np.where(e < mu, 1.0, np.where(e > mu, 0.0, 0.5))
    return 0.5 * (1.0 - np.tanh((e - mu) / (2.0 * kT)))


def density_exact(H: np.ndarray, b, C, mu: float, kT: float) -> np.ndarray:
    """rho_m = sum_alpha f(lambda_alpha) (C_m^T phi_alpha)(phi_alpha^T b): the
    density matrix of Eq. densityM-1 (Fermi-weighted eigenstates, the
    zero-broadening limit of Eq. densityM) projected on C_m and b, by a dense
    symmetric eigendecomposition."""
    lam, phi = np.linalg.eigh(H)
    C = np.atleast_2d(np.asarray(C, dtype=np.complex128))
    return ((C @ phi) * fermi(lam, mu, kT)) @ (phi.T @ np.asarray(b, dtype=np.complex128))


def density_quadrature(G: np.ndarray, energies, mu: float, kT: float) -> np.ndarray:
    """Eq. densityM on a uniform real-axis grid: rho_m = -(1/pi) sum_k w_k
    f(e_k) Im G_m(e_k + i delta) with trapezoid weights w_k, given G[m, k]."""
    e = np.asarray(energies, dtype=np.float64)
    h = e[1] - e[0]
    w = np.full(e.size, h)
    w[0] = w[-1] = 0.5 * h
    return -(np.asarray(G).imag * (w * fermi(e, mu, kT))).sum(axis=-1) / np.pi
