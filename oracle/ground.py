"""Ground state and one-particle excitations of the many-electron problem.

TEST INFRASTRUCTURE ONLY: the tests and ``__graft_entry__.smoke()`` use it;
the product path never imports it and shares no code with it.

Sec. II.B of arXiv:0802.0748: the ground state is found by the Lanczos
method, whose basis loses orthogonality after a few steps, and is then
improved by the conjugate-gradient method used as inverse iteration; the two
are repeated until the residual norm is small enough.  The excitation
spectra then follow from the shifted solver applied to c|psi_0> and
c+|psi_0> (Sec. IV.B, ionization and affinity levels).

Plain NumPy in FP64; ``H`` is anything with ``@`` (a dense array or a
scipy.sparse matrix).

* ``lanczos_ground_state``  Lanczos (no reorthogonalization), lowest Ritz pair,
                            residual, CG inverse iteration, repeated (Sec. II.B)
* ``fermion_op``            c_{i s} or c+_{i s} between particle-number sectors,
                            from the Jordan-Wigner definition acting on
                            occupation patterns (Sec. IV.B's model)
* ``fermion_op_at``         selected entries of the same, one by one
* ``hubbard_rows_apply``    (H psi) on selected rows, from the operators
* ``krylov_sd``             Green's functions by subspace diagonalisation in the
                            Krylov subspace (Sec. III.B, Eq. Ham_in_KS)
* ``excitation_green``      <b|(z - H)^{-1}|b> by dense solves (Eq. gf)
* ``lehmann_green``         the same from the eigen-decomposition of H

Readings where the paper is silent: the Lanczos basis is not
reorthogonalized (the paper's remedy for the lost orthogonality is the
inverse iteration); each cycle runs at most ``m`` Lanczos steps from the
current vector and restarts from the improved one; the inverse-iteration
shift is sigma = theta - ||r|| (theta the Rayleigh quotient, r = H psi -
theta psi), which lies below the lowest eigenvalue once psi is close to
the ground state, so that H - sigma is positive definite; the CG solve of
(H - sigma) y = psi starts from y = 0 and stops after ``cg_steps`` steps, at
a relative residual of 1e-10, or when p^T (H - sigma) p <= 0; the last
cycle runs no inverse iteration, so that the returned vector is the one whose
energy and residual are reported.
"""
from __future__ import annotations

import numpy as np

CG_RTOL = 1e-10


def _lanczos(H, v0, m):
    """m Lanczos steps from v0 (Sec. II.B): returns (alpha, beta, V) with
    H V_k = V_k T_k + beta_{k-1} v_k e_k^T, T_k = tridiag(beta, alpha, beta).
    Stops early when beta_j vanishes (an invariant subspace)."""
    n = v0.shape[0]
    V = np.zeros((m, n))
    V[0] = v0 / np.linalg.norm(v0)
    alpha, beta = [], []
    tnorm = 0.0
    for j in range(m):
        w = H @ V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        a = float(V[j] @ w)
        w = w - a * V[j]
        b = float(np.linalg.norm(w))
        alpha.append(a)
        beta.append(b)
        tnorm = max(tnorm, abs(a) + b + (beta[j - 1] if j > 0 else 0.0))
        if j + 1 == m or b <= 1e-12 * tnorm:
            break
        V[j + 1] = w / b
    k = len(alpha)
    return np.array(alpha), np.array(beta[:k - 1]), V[:k]


def _cg_inverse_step(H, psi, sigma, cg_steps):
    """CG on (H - sigma) y = psi from y = 0 (inverse iteration by CG, Sec. II.B)."""
    y = np.zeros_like(psi)
    r = psi.copy()
    p = psi.copy()
    rr = float(r @ r)
    rr0 = rr
    for _ in range(cg_steps):
        q = H @ p - sigma * p
        pq = float(p @ q)
        if not (pq > 0.0) or not np.isfinite(pq):
            break
        g = rr / pq
        y = y + g * p
        r = r - g * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        if rr <= CG_RTOL * CG_RTOL * rr0:
            break
    return y


class GroundState:
    def __init__(self, energy, psi, resid, status, lanczos_steps, cg_steps, cycles):
        self.energy = energy
        self.psi = psi
        self.resid = resid
        self.status = status            # 0 converged, 1 not converged
        self.lanczos_steps = lanczos_steps
        self.cg_steps = cg_steps
        self.cycles = cycles


def lanczos_ground_state(H, v0, m=60, cg_steps=0, max_cycles=50, tol=1e-10):
    """Lowest eigenpair of the real symmetric H by the Lanczos / CG-inverse-
    iteration cycle of Sec. II.B.  Converged when ||H psi - E psi||_2 <= tol
    with ||psi||_2 = 1 and E = psi^T H psi."""
    psi = np.asarray(v0, dtype=np.float64)
    psi = psi / np.linalg.norm(psi)
    nl = ncg = 0
    E = res = float("nan")
    for cycle in range(1, max_cycles + 1):
        alpha, beta, V = _lanczos(H, psi, m)
        nl += alpha.size
        T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
        evals, evecs = np.linalg.eigh(T)
        psi = evecs[:, 0] @ V
        psi = psi / np.linalg.norm(psi)
        Hpsi = H @ psi
        E = float(psi @ Hpsi)
        res = float(np.linalg.norm(Hpsi - E * psi))
        if res <= tol:
            return GroundState(E, psi, res, 0, nl, ncg, cycle)
        if cg_steps > 0 and cycle < max_cycles:
            y = _cg_inverse_step(H, psi, E - res, cg_steps)
            ncg += cg_steps
            ny = float(np.linalg.norm(y))
            if ny > 0.0 and np.isfinite(ny):
                psi = y / ny
    return GroundState(E, psi, res, 1, nl, ncg, max_cycles)


# --------------------------------------------------------------------------
# one-particle operators between sectors (Jordan-Wigner on occupation patterns)
# --------------------------------------------------------------------------

def _sector(L, k):
    """L-bit strings with k ones in ascending numeric order (bit i = site i)."""
    return [s for s in range(1 << L) if bin(s).count("1") == k]


def fermion_op(L, n_up, n_dn, site, spin, create, psi):
    """c_{site,spin} psi (create=False) or c+_{site,spin} psi (create=True).

    psi lives in the sector (n_up, n_dn) with basis index
    pos(up string) * D_dn + pos(down string), pos = position among the
    same-popcount strings in ascending order.  Modes are ordered all up
    sites (0..L-1) then all down sites (L..2L-1); c_m = Z x ... x Z x a
    (Jordan-Wigner), so acting on an occupation pattern it gives the sign
    (-1)^(number of occupied modes before m).  Returns the vector in the
    target sector (n_up -+ 1 or n_dn -+ 1)."""
    d = 1 if create else -1
    tu, td = (n_up + d, n_dn) if spin == 0 else (n_up, n_dn + d)
    if min(tu, td) < 0 or max(tu, td) > L:
        raise ValueError("no target sector")
    ups, dns = _sector(L, n_up), _sector(L, n_dn)
    tups, tdns = _sector(L, tu), _sector(L, td)
    pos_u = {s: i for i, s in enumerate(tups)}
    pos_d = {s: i for i, s in enumerate(tdns)}
    out = np.zeros(len(tups) * len(tdns), dtype=np.result_type(psi, np.float64))
    m = site + spin * L
    for iu, u in enumerate(ups):
        for idn, dd in enumerate(dns):
            occ = [(u >> i) & 1 for i in range(L)] + [(dd >> i) & 1 for i in range(L)]
            if occ[m] == (1 if create else 0):
                continue
            sign = -1.0 if sum(occ[:m]) % 2 else 1.0
            occ[m] ^= 1
            nu = sum(occ[i] << i for i in range(L))
            nd = sum(occ[L + i] << i for i in range(L))
            out[pos_u[nu] * len(tdns) + pos_d[nd]] += sign * psi[iu * len(dns) + idn]
    return out


def _flip(occ, m, create):
    """c_m (create=False) or c+_m on an occupation tuple: (sign, new tuple), or
    None when the mode is already empty (full).  Sign (-1)^(occupied modes
    before m), the Jordan-Wigner string."""
    if occ[m] == (1 if create else 0):
        return None
    sign = -1.0 if sum(occ[:m]) % 2 else 1.0
    new = list(occ)
    new[m] ^= 1
    return sign, tuple(new)


def fermion_op_at(L, n_up, n_dn, site, spin, create, psi, targets):
    """Entries ``targets`` of fermion_op(...): for each target basis state, the
    source state is the target with the mode flipped back, and the entry is the
    operator's sign on the source pattern times psi[source] (0 if the target
    has the mode in the wrong state).  For checks at sizes where the whole
    vector is out of reach."""
    d = 1 if create else -1
    tu, td = (n_up + d, n_dn) if spin == 0 else (n_up, n_dn + d)
    ups, dns = _sector(L, n_up), _sector(L, n_dn)
    tups, tdns = _sector(L, tu), _sector(L, td)
    pos_u = {s: i for i, s in enumerate(ups)}
    pos_d = {s: i for i, s in enumerate(dns)}
    m = site + spin * L
    out = np.zeros(len(targets), dtype=np.float64)
    for k, t in enumerate(targets):
        u, dd = tups[int(t) // len(tdns)], tdns[int(t) % len(tdns)]
        occ = tuple([(u >> i) & 1 for i in range(L)] + [(dd >> i) & 1 for i in range(L)])
        back = _flip(occ, m, not create)           # the source pattern
        if back is None:
            continue
        src = back[1]
        sign = _flip(src, m, create)[0]
        nu = sum(src[i] << i for i in range(L))
        nd = sum(src[L + i] << i for i in range(L))
        out[k] = sign * psi[pos_u[nu] * len(dns) + pos_d[nd]]
    return out


def hubbard_rows_apply(L, n_up, n_dn, t, U, V, periodic, psi, rows):
    """(H psi)[rows] for the extended Hubbard ring of Sec. IV.B,
    H = -t sum_{<ij>,s} (c+_is c_js + h.c.) + U sum_i n_iu n_id + V sum_<ij> n_i n_j,
    each row from the operators acting on that basis pattern (H is real
    symmetric, so row s is H|s> read in the basis).  Bonds (i, i+1), and
    (L-1, 0) on a ring of L >= 3."""
    ups, dns = _sector(L, n_up), _sector(L, n_dn)
    pos_u = {s: i for i, s in enumerate(ups)}
    pos_d = {s: i for i, s in enumerate(dns)}
    bonds = [(i, i + 1) for i in range(L - 1)] + ([(L - 1, 0)] if periodic and L >= 3 else [])
    out = np.zeros(len(rows), dtype=np.float64)
    for k, r in enumerate(rows):
        u, dd = ups[int(r) // len(dns)], dns[int(r) % len(dns)]
        occ = tuple([(u >> i) & 1 for i in range(L)] + [(dd >> i) & 1 for i in range(L)])
        nsite = [occ[i] + occ[L + i] for i in range(L)]
        acc = (U * sum(occ[i] * occ[L + i] for i in range(L)) + V * sum(nsite[i] * nsite[j] for i, j in bonds)) \
            * psi[int(r)]
        for i, j in bonds:
            for sp in range(2):
                for a, b in ((i + sp * L, j + sp * L), (j + sp * L, i + sp * L)):
                    s1 = _flip(occ, b, False)              # c_b
                    if s1 is None:
                        continue
                    s2 = _flip(s1[1], a, True)             # c+_a
                    if s2 is None:
                        continue
                    o = s2[1]
                    nu = sum(o[x] << x for x in range(L))
                    nd = sum(o[L + x] << x for x in range(L))
                    acc += -t * s1[0] * s2[0] * psi[pos_u[nu] * len(dns) + pos_d[nd]]
        out[k] = acc
    return out


class KrylovSD:
    def __init__(self, G, ritz, weight, nu):
        self.G = G              # [M][K]
        self.ritz = ritz        # [nu] eigenvalues of T, ascending
        self.weight = weight    # [M][nu] (c_m^T w_a)(w_a^T b)
        self.nu = nu            # Lanczos steps done


def krylov_sd(H, b, nu, shifts, C):
    """Subspace diagonalisation in the Krylov subspace K_nu(H, b) (Sec. III.B,
    Eq. Ham_in_KS): the reduced Hamiltonian in the Lanczos basis v_0..v_{nu-1}
    (no reorthogonalization) is the tridiagonal T; its eigenpairs (e_a, s_a)
    give approximate eigenvectors w_a = sum_j s_a(j) v_j, and
        G_m(z) = sum_a (c_m^T w_a)(w_a^T b) / (z - e_a),
    with w_a^T b = ||b|| s_a(0).  C: [M][N] real projection vectors."""
    b = np.asarray(b, dtype=np.float64)
    C = np.atleast_2d(np.asarray(C, dtype=np.float64))
    alpha, beta, V = _lanczos(H, b, nu)
    T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    e, S = np.linalg.eigh(T)
    P = C @ V.T                                   # [M][k]: c_m^T v_j
    weight = (P @ S) * (np.linalg.norm(b) * S[0])[None, :]
    shifts = np.asarray(shifts, dtype=np.complex128)
    G = weight @ (1.0 / (shifts[None, :] - e[:, None]))
    return KrylovSD(G, e, weight, alpha.size)


def excitation_green(H, b, shifts):
    """G(z_k) = b^T (z_k - H)^{-1} b by dense solves (Eq. gf with c = b real)."""
    H = np.asarray(H.todense() if hasattr(H, "todense") else H, dtype=np.float64)
    n = H.shape[0]
    out = np.empty(len(shifts), dtype=np.complex128)
    for k, z in enumerate(shifts):
        x = np.linalg.solve(z * np.eye(n) - H, b.astype(np.complex128))
        out[k] = b @ x
    return out


def lehmann_green(H, b, shifts):
    """The same G from the eigen-decomposition: sum_n |<n|b>|^2 / (z - E_n)."""
    H = np.asarray(H.todense() if hasattr(H, "todense") else H, dtype=np.float64)
    E, U = np.linalg.eigh(H)
    w = (U.T @ b) ** 2
    return np.array([np.sum(w / (z - E)) for z in shifts])


def free_fermion_ground_energy(L, n_up, n_dn, t):
    """Lowest many-body energy of -t sum (c+_i c_{i+1} + h.c.) on a periodic
    ring: the n_up and n_dn lowest of -2 t cos(2 pi m / L)."""
    eps = np.sort(-2.0 * t * np.cos(2 * np.pi * np.arange(L) / L))
    return float(eps[:n_up].sum() + eps[:n_dn].sum())


def occupations(L, n_up, n_dn, psi):
    """<n_{i s}> for every site and spin: sum of |psi|^2 over basis states
    whose string has bit i set.  Returns [2][L]."""
    ups, dns = _sector(L, n_up), _sector(L, n_dn)
    p2 = np.abs(np.asarray(psi).reshape(len(ups), len(dns))) ** 2
    out = np.zeros((2, L))
    for i in range(L):
        mu = np.array([(u >> i) & 1 for u in ups], dtype=float)
        md = np.array([(d >> i) & 1 for d in dns], dtype=float)
        out[0, i] = float(mu @ p2.sum(axis=1))
        out[1, i] = float(md @ p2.sum(axis=0))
    return out


__all__ = ["krylov_sd", "KrylovSD", "lanczos_ground_state", "fermion_op", "fermion_op_at", "hubbard_rows_apply", "excitation_green", "lehmann_green",
           "free_fermion_ground_energy", "occupations", "GroundState", "CG_RTOL"]
