"""Jordan-Wigner Fock-space Hamiltonian for a handful of orbitals (2n <= 8 modes).

Test infrastructure: only the tests import this module.

Builds the fermionic modes as explicit 2^(2n) x 2^(2n) matrices with the
Jordan-Wigner mapping of the paper's Methods ("Mapping fermionic Hamiltonians
to the qubits": a_j -> (prod_{i<j} sigma^z_i) sigma^-_j), with the paper's
interleaved mode order (spatial orbital i -> spin-up mode 2i, spin-down mode
2i+1; the paper counts from 1), and forms the second-quantized electronic
Hamiltonian directly from its definition:

    H = sum_{pq,s} h_pq a+_{ps} a_{qs}
      + 1/2 sum_{pqrs,s,t} (pq|rs) a+_{ps} a+_{rt} a_{st} a_{qs}.

Basis state |x>, x an integer with bit j = occupation of mode j, is the product
of creators in ascending mode order acting on the vacuum.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = ["annihilators", "hamiltonian", "number_ops", "sector_map"]


def annihilators(nmodes: int):
    """Jordan-Wigner annihilators a_0 .. a_{nmodes-1} (sparse CSR)."""
    dim = 1 << nmodes
    ops = []
    for j in range(nmodes):
        rows, cols, vals = [], [], []
        for x in range(dim):
            if (x >> j) & 1:
                parity = bin(x & ((1 << j) - 1)).count("1") & 1
                rows.append(x ^ (1 << j))
                cols.append(x)
                vals.append(-1.0 if parity else 1.0)
        ops.append(sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim)))
    return ops


def mode(p: int, spin: int) -> int:
    """Interleaved mode index of spatial orbital p, spin 0 (up) / 1 (down)."""
    return 2 * p + spin


def hamiltonian(h1: np.ndarray, eri: np.ndarray):
    n = h1.shape[0]
    nm = 2 * n
    a = annihilators(nm)
    ad = [m.T.tocsr() for m in a]
    dim = 1 << nm
    H = sp.csr_matrix((dim, dim))
    for s in range(2):
        for p in range(n):
            for q in range(n):
                if h1[p, q] != 0.0:
                    H = H + h1[p, q] * (ad[mode(p, s)] @ a[mode(q, s)])
    for s in range(2):
        for t in range(2):
            for p in range(n):
                for q in range(n):
                    A = a[mode(q, s)]
                    for r in range(n):
                        B = ad[mode(p, s)] @ ad[mode(r, t)]
                        for x in range(n):
                            v = eri[p, q, r, x]
                            if v != 0.0:
                                H = H + 0.5 * v * (B @ (a[mode(x, t)] @ A))
    return H.toarray()


def number_ops(n: int):
    """(N, S_z) as dense diagonal matrices over 2n interleaved modes."""
    nm = 2 * n
    dim = 1 << nm
    N = np.zeros(dim)
    Sz = np.zeros(dim)
    for x in range(dim):
        for p in range(n):
            up = (x >> mode(p, 0)) & 1
            dn = (x >> mode(p, 1)) & 1
            N[x] += up + dn
            Sz[x] += 0.5 * (up - dn)
    return np.diag(N), np.diag(Sz)


def sector_map(n: int, masks_a, masks_b):
    """For each determinant (I_a, I_b) in alpha-major order: its Fock index and
    the sign relating the alpha-first creator order to the interleaved one.

    The alpha-first state puts all alpha creators (ascending) left of all beta
    creators (ascending); moving each beta creator of orbital b rightwards past
    the alpha creators of orbitals a > b yields the interleaved order, one
    transposition each.
    """
    idx = []
    sgn = []
    for Ia in masks_a:
        for Ib in masks_b:
            x = 0
            swaps = 0
            for p in range(n):
                if (Ia >> p) & 1:
                    x |= 1 << mode(p, 0)
                if (Ib >> p) & 1:
                    x |= 1 << mode(p, 1)
                    swaps += bin(int(Ia) >> (p + 1)).count("1")
            idx.append(x)
            sgn.append(-1.0 if swaps & 1 else 1.0)
    return np.array(idx), np.array(sgn)
