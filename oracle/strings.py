"""Occupation strings and single-excitation tables, by brute force.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this package.

The determinant basis of a fixed (N_alpha, N_beta) sector -- the sector the
paper's number-conserving sampler restricts itself to (Results, "Parallel
sampling", the constraint on the conditionals) -- is a product of alpha and beta
occupation strings.  A string with m electrons in n spatial orbitals is an n-bit
mask with popcount m; bit p set means orbital p occupied.  Here every such mask
is enumerated by scanning all 2^n integers, and its rank is its position in
ascending integer order.

A string's state is the product of creators in ascending orbital order acting on
the vacuum.  The spin-summed excitation E_pq = sum_sigma a^dag_{p sigma}
a_{q sigma} of the paper's Methods Hamiltonian acts on one spin's string as
a^dag_p a_q.  The table lists, for every string I and every (p, q) with
a^dag_p a_q |I> != 0, the target rank J, the pair index p*n+q and the fermionic
sign, in this order: I ascending; q over the occupied orbitals ascending; p over
{q} union (vacant orbitals), ascending.  The sign is obtained here by applying
the two operators one after the other with the Jordan-Wigner rule (a creator or
annihilator at p picks up (-1)^(number of occupied orbitals below p)).
"""
from __future__ import annotations

import numpy as np

__all__ = ["enumerate_strings", "rank_lookup", "apply_annihilator", "apply_creator",
           "excitation_table", "n_exc"]


def enumerate_strings(norb: int, nelec: int) -> np.ndarray:
    """All n-bit masks with ``nelec`` bits set, ascending (brute force)."""
    out = [x for x in range(1 << norb) if bin(x).count("1") == nelec]
    return np.array(out, dtype=np.int64)


def rank_lookup(norb: int, masks: np.ndarray) -> np.ndarray:
    """Dense mask -> rank table of size 2^n (-1 for masks outside the sector)."""
    lut = np.full(1 << norb, -1, dtype=np.int64)
    lut[masks] = np.arange(len(masks))
    return lut


def apply_annihilator(mask: int, p: int):
    """a_p |mask>  ->  (new_mask, sign) or (None, 0) if orbital p is empty."""
    if not (mask >> p) & 1:
        return None, 0
    below = bin(mask & ((1 << p) - 1)).count("1")
    return mask & ~(1 << p), (-1 if below & 1 else 1)


def apply_creator(mask: int, p: int):
    """a^dag_p |mask>  ->  (new_mask, sign) or (None, 0) if orbital p is full."""
    if (mask >> p) & 1:
        return None, 0
    below = bin(mask & ((1 << p) - 1)).count("1")
    return mask | (1 << p), (-1 if below & 1 else 1)


def n_exc(norb: int, nelec: int) -> int:
    """Entries per string: m occupied q times (n-m vacant p + the diagonal p=q)."""
    return nelec * (norb - nelec + 1)


def excitation_table(norb: int, nelec: int):
    """(masks, tgt[N_s, n_exc] int32, pq[N_s, n_exc] uint16, sgn[N_s, n_exc] int8)."""
    masks = enumerate_strings(norb, nelec)
    lut = rank_lookup(norb, masks)
    ns = len(masks)
    ne = n_exc(norb, nelec)
    tgt = np.zeros((ns, ne), dtype=np.int32)
    pq = np.zeros((ns, ne), dtype=np.uint16)
    sgn = np.zeros((ns, ne), dtype=np.int8)
    for i, I in enumerate(masks.tolist()):
        k = 0
        occ = [q for q in range(norb) if (I >> q) & 1]
        vac = [p for p in range(norb) if not (I >> p) & 1]
        for q in occ:
            for p in sorted([q] + vac):
                m1, s1 = apply_annihilator(I, q)
                m2, s2 = apply_creator(m1, p)
                tgt[i, k] = lut[m2]
                pq[i, k] = p * norb + q
                sgn[i, k] = s1 * s2
                k += 1
        assert k == ne
    return masks, tgt, pq, sgn
