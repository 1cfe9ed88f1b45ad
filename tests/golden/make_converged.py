"""Writes the converged Green's functions of the full-size workloads that the
GPU parity tests and the benchmark compare against.

Every stored value comes from the CPU oracle alone (``oracle.shifted_cocg``:
plain FP64 textbook shifted COCG with full per-shift vectors, Sec. III.C of
arXiv:0802.0748), run to a relative residual of 1e-12 on a seeded subset of
each workload's shifts: the seed shift of the whole list (the oracle's seed
rule) plus 16 others drawn with numpy's PCG64.  The inputs come from
``paper_0802_0748_gb300.inputs`` (seeded synthesis only, no solver
arithmetic).  The exact shifts are stored beside G, together with checksums
of H and b, so a consumer can check that it regenerated the same problem.

Usage (each workload takes minutes to hours of CPU time; OMP_NUM_THREADS
sets the oracle's thread count):

    python tests/golden/make_converged.py anderson   # 64^3 x 4, 512 shifts, eta 1e-3
    python tests/golden/make_converged.py hubbard    # 14-site ring, 128 shifts, eta 0.05
    python tests/golden/make_converged.py batch      # 32^3 x 4, 4 of the 256 unit rhs, eta 1e-2
    python tests/golden/make_converged.py adjoint    # 24^3 x 4 gradient dL/dH, 128 shifts, eta 0.02

The adjoint file holds the oracle gradient (oracle.grad_from_vectors on the
oracle's full per-shift solutions, residual 1e-13) of L = sum_k w_k Im G_00(z_k)
on a seeded sample of the stored entries plus the entries of largest |g|.
"""
from __future__ import annotations

import json
import sys
import time
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
ROOT = HERE.parent.parent
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_0802_0748_gb300 import inputs  # noqa: E402

TOL = 1e-12
MAX_ITER = 600000
N_EXTRA = 16
BATCH_RHS = (0, 77, 150, 255)
ADJOINT_BOUNDS = (-6.0, 6.4)     # the bounds the gradient benchmark and tests use


def shift_subset(shifts: np.ndarray, draw_seed: int) -> tuple[np.ndarray, int]:
    """Indices (ascending) of the seed shift plus N_EXTRA seeded others, and
    the position of the seed shift among them."""
    seed = oracle.default_seed(shifts)
    others = np.setdiff1d(np.arange(shifts.size), [seed])
    pick = np.random.default_rng(draw_seed).choice(others, size=N_EXTRA, replace=False)
    idx = np.sort(np.concatenate([[seed], pick])).astype(np.int64)
    return idx, int(np.where(idx == seed)[0][0])


def checksum(a: np.ndarray) -> list[float]:
    """Order-independent fingerprint of an array: sum and sum of squares of its
    real view (enough to tell a regenerated input from a different one)."""
    v = np.asarray(a).view(np.float64) if np.iscomplexobj(a) else np.asarray(a, dtype=np.float64)
    return [float(np.sum(v)), float(np.sum(v * v))]


def cplx_list(a) -> list[list[float]]:
    return [[float(x.real), float(x.imag)] for x in np.asarray(a).ravel()]


def solve(rowptr, col, val, shifts, b, idx, seed_pos, *, proj_idx=None, proj_vec=None) -> dict:
    t0 = time.time()
    res = oracle.shifted_cocg(rowptr, col, val, shifts[idx], b, proj_idx=proj_idx, proj_vec=proj_vec,
                              tol=TOL, max_iter=MAX_ITER, seed=seed_pos)
    if res.status != oracle.OK:
        raise RuntimeError(f"oracle status {res.status} after {res.n_iter} iterations")
    return {"G": cplx_list(res.G[0]), "iters": [int(x) for x in res.iters], "n_iter": res.n_iter,
            "n_switch": res.n_switch, "resid_max": float(res.resid.max()), "cpu_seconds": time.time() - t0}


def make_anderson() -> dict:
    wl = inputs.workload("anderson", "full", bounds=inputs.ANDERSON64_BOUNDS)
    h = wl.csr
    idx, sp = shift_subset(wl.shifts, 22)
    out = {"workload": "anderson-64^3x4 seed 2, 512 shifts e_k + 1e-3 i over ANDERSON64_BOUNDS, "
                       "b = random_unit_complex(n, 2), c = conj(b)",
           "bounds": list(inputs.ANDERSON64_BOUNDS), "subset": idx.tolist(), "seed_in_subset": sp,
           "shifts": cplx_list(wl.shifts[idx]), "val_checksum": checksum(h.val), "b_checksum": checksum(wl.rhs[0])}
    out.update(solve(h.rowptr, h.col, h.val, wl.shifts, wl.rhs[0], idx, sp, proj_vec=wl.proj_vec))
    return out


def make_hubbard() -> dict:
    wl = inputs.workload("hubbard", "full")
    p = wl.hubbard
    rp, col, val = oracle.hubbard_csr(p["L"], p["n_up"], p["n_dn"], p["t"], p["U"], p["V"], p["periodic"])
    idx, sp = shift_subset(wl.shifts, 55)
    out = {"workload": "Hubbard ring L=14, 7 up 7 down, t=1 U=4 V=1 periodic, 128 shifts "
                       "linspace(-10, 20) + 0.05 i, b = random_unit_complex(n, 5), c = conj(b)",
           "subset": idx.tolist(), "seed_in_subset": sp, "shifts": cplx_list(wl.shifts[idx]),
           "b_checksum": checksum(wl.rhs[0])}
    out.update(solve(rp, col, val, wl.shifts, wl.rhs[0], idx, sp, proj_vec=wl.proj_vec))
    return out


def make_batch() -> dict:
    wl = inputs.workload("batch", "full", bounds=inputs.BATCH32_BOUNDS)
    h = wl.csr
    idx, sp = shift_subset(wl.shifts, 33)
    out = {"workload": "anderson-32^3x4 seed 3, 256 unit rhs e_j with projection e_j, 256 shifts "
                       "linspace over BATCH32_BOUNDS + 1e-2 i",
           "bounds": list(inputs.BATCH32_BOUNDS), "subset": idx.tolist(), "seed_in_subset": sp,
           "shifts": cplx_list(wl.shifts[idx]), "val_checksum": checksum(h.val), "rhs": {}}
    for j in BATCH_RHS:
        site = int(wl.proj_idx[j, 0])
        r = solve(h.rowptr, h.col, h.val, wl.shifts, wl.rhs[j], idx, sp, proj_idx=[site])
        r["site"] = site
        out["rhs"][str(j)] = r
    return out


def make_adjoint() -> dict:
    wl = inputs.workload("adjoint", "full", bounds=ADJOINT_BOUNDS)
    h = wl.csr
    t0 = time.time()
    res = oracle.shifted_cocg(h.rowptr, h.col, h.val, wl.shifts, wl.rhs[0], proj_idx=[0], tol=1e-13,
                              max_iter=MAX_ITER, want_x=True)
    if res.status != oracle.OK:
        raise RuntimeError(f"oracle status {res.status}")
    gbar = 1j * wl.weights
    g = oracle.grad_from_vectors(h.rowptr, h.col, res.X, res.X, gbar)   # c = b = e_0: y_k = x_k
    rng = np.random.default_rng(44)
    sample = rng.choice(h.nnz, size=4096, replace=False)
    top = np.argsort(np.abs(g))[::-1][:64]
    idx = np.unique(np.concatenate([sample, top])).astype(np.int64)
    return {"workload": "anderson-24^3x4 seed 4, b = c = e_0, 128 shifts linspace over ADJOINT_BOUNDS + 0.02 i, "
                        "L = sum_k w_k Im G_00(z_k), w = workload weights",
            "bounds": list(ADJOINT_BOUNDS), "shifts": cplx_list(wl.shifts), "val_checksum": checksum(h.val),
            "weights": [float(x) for x in wl.weights], "g_inf_norm": float(np.abs(g).max()),
            "entries": idx.tolist(), "g": [float(x) for x in g[idx]], "n_iter": res.n_iter,
            "resid_max": float(res.resid.max()), "cpu_seconds": time.time() - t0, "tol": 1e-13}


MAKERS = {"anderson": (make_anderson, "anderson64x4_converged.json"),
          "hubbard": (make_hubbard, "hubbard14_converged.json"),
          "batch": (make_batch, "batch32x4_converged.json"),
          "adjoint": (make_adjoint, "adjoint24x4_gradient.json")}


def main(argv):
    names = argv[1:] or list(MAKERS)
    for name in names:
        fn, fname = MAKERS[name]
        data = fn()
        data.setdefault("tol", TOL)
        data.update({"oracle": "oracle.shifted_cocg (FP64, full per-shift vectors)",
                     "command": f"python tests/golden/make_converged.py {name}"})
        (HERE / fname).write_text(json.dumps(data, indent=1) + "\n")
        print(name, "done", data.get("n_iter"), flush=True)


if __name__ == "__main__":
    main(sys.argv)
