"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and assembles the input arrays of the
workloads; it holds none of the method's arithmetic (no Hamiltonian, no
excitation tables, no recursion).  Both the CPU oracle and the CUDA path read
their inputs from here, so that they see bit-identical integrals and states.

Integral recipe (one draw order, NumPy PCG64 ``default_rng(seed)``):

1. ``h1``: diagonal = ``linspace(-2, 1, n)``; one n x n draw of N(0, 0.05^2),
   strict upper triangle mirrored onto the lower one.
2. For Q = 0 .. nchol-1: one n x n draw of N(0, 0.1^2), upper triangle
   (diagonal included) mirrored -> symmetric L_Q.  The two-electron integrals
   in chemist order are (pq|rs) = sum_Q L_Q[p,q] L_Q[r,s]; by construction they
   have the 8-fold permutational symmetry and are positive semi-definite as an
   n^2 x n^2 matrix, like a Cholesky-decomposed molecular ERI tensor.
3. Dipole integrals d^x, d^y, d^z: three n x n draws of N(0, 0.3^2), upper
   triangle (diagonal included) mirrored.

These stand in for the STO-3G molecular integrals of the paper's Table 1 and
Fig. 3 molecules, which are not available here.
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Integrals",
    "integrals",
    "random_state",
    "WORKLOADS",
    "workload",
    "serving_stream",
    "array_digest",
]


@dataclass
class Integrals:
    """Molecular-integral stand-ins for one seeded synthetic system."""

    norb: int
    nalpha: int
    nbeta: int
    h1: np.ndarray          # (n, n) float64, symmetric
    eri: np.ndarray         # (n, n, n, n) float64, chemist (pq|rs)
    dipole: np.ndarray      # (3, n, n) float64, symmetric per component
    seed: int
    nchol: int
    meta: dict = field(default_factory=dict)


def _mirror_upper(m: np.ndarray, include_diag: bool) -> np.ndarray:
    k = 0 if include_diag else 1
    u = np.triu(m, k)
    out = u + np.triu(m, 1).T
    return out


def integrals(norb: int, nalpha: int, nbeta: int, seed: int,
              nchol: int | None = None) -> Integrals:
    """Draw h1, (pq|rs) and d^{x,y,z} for ``norb`` spatial orbitals.

    ``nchol`` defaults to 2*norb (16 vectors at 8 orbitals, 24 at 12, 32 at
    16, 36 at 18).
    """
    if nchol is None:
        nchol = 2 * norb
    n = norb
    rng = np.random.default_rng(seed)
    off = rng.normal(0.0, 0.05, size=(n, n))
    h1 = _mirror_upper(off, include_diag=False)
    h1[np.diag_indices(n)] = np.linspace(-2.0, 1.0, n)
    L = np.empty((nchol, n, n))
    for q in range(nchol):
        L[q] = _mirror_upper(rng.normal(0.0, 0.1, size=(n, n)), include_diag=True)
    eri = np.einsum("qij,qkl->ijkl", L, L, optimize=True)
    dip = np.empty((3, n, n))
    for c in range(3):
        dip[c] = _mirror_upper(rng.normal(0.0, 0.3, size=(n, n)), include_diag=True)
    return Integrals(norb=n, nalpha=nalpha, nbeta=nbeta, h1=h1, eri=eri,
                     dipole=dip, seed=seed, nchol=nchol)


def random_state(dim: int, seed: int) -> np.ndarray:
    """A seeded, normalised FP64 vector of length ``dim`` (standard normal draws)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(dim)
    v /= np.linalg.norm(v)
    return v


def _binom(n: int, k: int) -> int:
    return math.comb(n, k)


# The five workloads of the benchmark suite.  Names describe the system.
WORKLOADS = {
    "fci8o8e": dict(norb=8, nalpha=4, nbeta=4, seed=2506071, nmoments=256,
                    npoints=2048, ncol=3, precision="fp64"),
    "fci12o12e": dict(norb=12, nalpha=6, nbeta=6, seed=2506072, nmoments=1024,
                      npoints=2048, ncol=3, precision="fp32"),
    "fci14o14e": dict(norb=14, nalpha=7, nbeta=7, seed=2506074, nmoments=1024,
                      npoints=2048, ncol=3, precision="mixed"),
    "fci16o16e": dict(norb=16, nalpha=8, nbeta=8, seed=2506073, nmoments=2048,
                      npoints=2048, ncol=1, precision="mixed"),
    "fci18o18e": dict(norb=18, nalpha=9, nbeta=9, seed=2506075, nmoments=1024,
                      npoints=2048, ncol=1, precision="mixed"),
}
for _k, _w in WORKLOADS.items():
    _w["dim"] = _binom(_w["norb"], _w["nalpha"]) * _binom(_w["norb"], _w["nbeta"])
    _w["nchol"] = 2 * _w["norb"]


def workload(name: str) -> dict:
    return dict(WORKLOADS[name])


def serving_stream(nreq: int = 64, rate_hz: float | None = None,
                   arrival_seed: int = 2506199, first_seed: int = 2506100,
                   sizes=((10, 5), (12, 6), (14, 7)),
                   moment_choices=(512, 768, 1024, 1280, 1536, 1792, 2048)):
    """Request list for the serving workload.

    Each request r draws its size uniformly from ``sizes`` (norb, electrons per
    spin) and its moment count uniformly from ``moment_choices`` with
    ``default_rng(first_seed + r)``; its integrals use seed ``first_seed + r``.
    Arrival times are a Poisson process of rate ``rate_hz`` drawn from
    ``default_rng(arrival_seed)`` (all at t=0 when ``rate_hz`` is None).
    """
    reqs = []
    arr = np.random.default_rng(arrival_seed)
    t = 0.0
    for r in range(nreq):
        rr = np.random.default_rng(first_seed + r)
        norb, ne = sizes[int(rr.integers(len(sizes)))]
        nm = int(moment_choices[int(rr.integers(len(moment_choices)))])
        if rate_hz is not None:
            t += float(arr.exponential(1.0 / rate_hz))
        reqs.append(dict(id=r, norb=norb, nalpha=ne, nbeta=ne, seed=first_seed + r,
                         nmoments=nm, arrival_s=t))
    return reqs


def array_digest(*arrays: np.ndarray) -> str:
    """SHA-256 over the raw little-endian bytes of the given arrays."""
    h = hashlib.sha256()
    for a in arrays:
        a = np.ascontiguousarray(a)
        h.update(str(a.dtype).encode())
        h.update(str(a.shape).encode())
        h.update(a.astype(a.dtype.newbyteorder("<"), copy=False).tobytes())
    return h.hexdigest()
