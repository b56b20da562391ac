"""CPU FP64 oracle for the KPM dipole-spectrum hot path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import, call, link or execute anything in this
package.  The product path (the CUDA library and its binding) never does; it
shares no code, header, table or constant with this package.  The only common
dependency is the seeded input generator ``synthetic``, which holds none of the
method's arithmetic.

Contents (every function cites the paper passage it follows):

* ``strings``     -- brute-force occupation strings and single-excitation tables.
* ``hamiltonian`` -- determinant-pair Slater-Condon H and dipole (C, ``sc.c``),
                     and an operator-by-operator NumPy form pinned to it.
* ``fock``        -- Jordan-Wigner Fock-space H for <= 4 spatial orbitals.
* ``kpm``         -- recursion and doubling moments, eigenpair moments,
                     Jackson kernel, spectrum by direct cosine sums.

Pins are in ``tests/test_oracle_*.py`` (run with ``-m "not gpu"``).  Parity of
every function is pinned there; nothing here is "parity unpinned".
"""
from __future__ import annotations

import numpy as np

from . import fock, hamiltonian, kpm, strings  # noqa: F401
from .hamiltonian import OperatorForm, SlaterCondon, build  # noqa: F401

__all__ = ["strings", "hamiltonian", "fock", "kpm", "SlaterCondon", "OperatorForm",
           "build", "ground_state", "spectral_bounds"]


def ground_state(op, dim: int, dense_limit: int = 6000, tol: float = 1e-12, seed: int = 7):
    """(E_0, |0>) of H.  Dense eigh up to ``dense_limit``, else ARPACK (Lanczos)
    on the matrix-free operator ``op(v) = H v``.  The paper's FCI baselines use
    Lanczos for the low eigenpairs (Results, absorption spectra of H2O/NH3)."""
    if dense_limit >= dim and hasattr(op, "__self__") and hasattr(op.__self__, "dense"):
        H = op.__self__.dense()
        w, v = np.linalg.eigh(H)
        return float(w[0]), v[:, 0].copy()
    import scipy.sparse.linalg as sla
    A = sla.LinearOperator((dim, dim), matvec=op, dtype=np.float64)
    v0 = np.random.default_rng(seed).standard_normal(dim)
    w, v = sla.eigsh(A, k=1, which="SA", tol=tol, v0=v0)
    return float(w[0]), v[:, 0].copy()


def spectral_bounds(op, dim: int, tol: float = 1e-10, seed: int = 11):
    """(E_min, E_max) of H by ARPACK, each widened by its Ritz residual norm."""
    import scipy.sparse.linalg as sla
    A = sla.LinearOperator((dim, dim), matvec=op, dtype=np.float64)
    v0 = np.random.default_rng(seed).standard_normal(dim)
    lo_w, lo_v = sla.eigsh(A, k=1, which="SA", tol=tol, v0=v0)
    hi_w, hi_v = sla.eigsh(A, k=1, which="LA", tol=tol, v0=v0)
    r_lo = np.linalg.norm(op(lo_v[:, 0]) - lo_w[0] * lo_v[:, 0])
    r_hi = np.linalg.norm(op(hi_v[:, 0]) - hi_w[0] * hi_v[:, 0])
    return float(lo_w[0] - r_lo), float(hi_w[0] + r_hi)
