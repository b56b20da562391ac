"""Writes tests/golden/moments_fci12o12e.json: the oracle's FP64 KPM moments of
the 12-orbital workload (6 alpha + 6 beta electrons, FCI dimension 853,776).

Inputs: the seeded integrals of the 12-orbital workload, a seeded normalised
state psi (``synthetic.random_state(dim, 2506172)``), and the x, y, z dipole
components alpha_0 = mu_c psi.  Spectral bounds from ARPACK on the oracle's
Slater-Condon row-pull, each widened by its Ritz residual, then a, b with
eps = 0.01.  Moments: 1024 per component by the Methods recursion and doubling
identities (``oracle.kpm.moments_recursion_block``), H applied by the oracle's
determinant-pair row-pull.  Calls only ``synthetic`` and ``oracle``; never the
CUDA library.  Run from the repository root (about half an hour on 8 cores):
    python tests/golden/make_moments_12o.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthetic  # noqa: E402
from oracle import kpm  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
STATE_SEED = 2506172
NMOMENTS = 1024


def main():
    w = synthetic.workload("fci12o12e")
    n, na, nb = w["norb"], w["nalpha"], w["nbeta"]
    I = synthetic.integrals(n, na, nb, w["seed"])
    sc = oracle.SlaterCondon(I.h1, I.eri, n, na, nb)
    t0 = time.time()
    emin, emax = oracle.spectral_bounds(sc.sigma, sc.dim, tol=1e-9)
    t_bounds = time.time() - t0
    a, b = kpm.scale_from_bounds(emin, emax)
    psi = synthetic.random_state(sc.dim, STATE_SEED)
    A0 = np.stack([sc.dipole(I.dipole[c], psi) for c in range(3)])
    t0 = time.time()
    mu = kpm.moments_recursion_block(sc.sigma_block, A0, a, b, NMOMENTS)
    t_mom = time.time() - t0
    out = {
        "workload": "fci12o12e", "norb": n, "nalpha": na, "nbeta": nb, "dim": sc.dim,
        "integral_seed": w["seed"], "state_seed": STATE_SEED,
        "state": "synthetic.random_state(dim, state_seed)", "components": "x, y, z",
        "emin": emin, "emax": emax, "eps": 0.01, "a": a, "b": b, "nmoments": NMOMENTS,
        "moments": [[float(v) for v in row] for row in mu],
        "oracle": "Slater-Condon row-pull (sc.c), FP64 recursion + doubling identities",
        "seconds": {"bounds": round(t_bounds, 1), "moments": round(t_mom, 1)},
    }
    with open(os.path.join(HERE, "moments_fci12o12e.json"), "w") as f:
        json.dump(out, f, indent=0)
    print("wrote moments_fci12o12e.json", out["seconds"])


if __name__ == "__main__":
    main()
