"""Batched recursion of several small molecules (kpm_moments_batch) through the C-ABI.

After each molecule's first step, every Chebyshev step of the whole batch is one
sigma launch and one update launch over a flattened grid.  Per molecule the
kernels run the same per-element arithmetic and the same fixed reduction grid as
the single-molecule path, so the moments must be identical (bit for bit) to
kpm_moments on each context; one molecule is also checked against the oracle's
FP64 recursion (1e-10 Omega_0, the FP64 moment tolerance of the parity tests).
"""
import numpy as np
import pytest

import oracle
import synthetic
from oracle import kpm as okpm

pytestmark = pytest.mark.gpu

# mixed sizes (one beyond the dense-eigensolver range), a one-determinant
# sector and a single-electron-per-spin case among them
MOLS = [(6, 3, 3), (8, 4, 4), (7, 2, 4), (5, 5, 0), (9, 4, 4), (4, 1, 1)]


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available()
    return _t


def _ab(I, n, na, nb):
    """Rescaling from the oracle's spectrum (dense below 4,900 determinants)."""
    sc = oracle.SlaterCondon(I.h1, I.eri, n, na, nb)
    if sc.dim <= 4900:
        E = np.linalg.eigvalsh(sc.dense())
        lo, hi = float(E[0]), float(E[-1])
    else:
        sc.csr()
        lo, hi = oracle.spectral_bounds(sc.sigma, sc.dim)
    if hi - lo < 1e-6 * max(1.0, abs(hi)):   # one determinant: any window around it
        lo, hi = lo - 1.0, hi + 1.0
    return okpm.scale_from_bounds(lo, hi)


def _batch(torch, prec, mols=MOLS, seed0=2506300):
    from paper_2506_07430_gb300 import KPM
    ks, psis, ab, ints = [], [], [], []
    for i, (n, na, nb) in enumerate(mols):
        I = synthetic.integrals(n, na, nb, seed=seed0 + i)
        k = KPM(I.h1, I.eri, I.dipole, n, na, nb, precision=prec)
        a, b = _ab(I, n, na, nb)
        psis.append(torch.tensor(synthetic.random_state(k.dim, 40 + i), device="cuda"))
        ks.append(k)
        ab.append((a, b))
        ints.append(I)
    return ks, psis, ab, ints


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("N", [64, 66, 2])
def test_batch_equals_single(torch, prec, N):
    """N = 64: 31 batched steps (odd: the rotating vectors end swapped); 66: even;
    2: no batched step at all."""
    from paper_2506_07430_gb300 import moments_batch
    ks, psis, ab, _ = _batch(torch, prec)
    a = [x[0] for x in ab]
    b = [x[1] for x in ab]
    got = moments_batch(ks, psis, 0b111, a, b, N)
    assert got.shape == (len(ks), 3, N)
    for i, k in enumerate(ks):
        one = k.moments(psis[i], 0b111, a[i], b[i], N)
        assert np.array_equal(got[i], one), (i, np.abs(got[i] - one).max())
    for k in ks:
        k.close()


def test_batch_against_oracle(torch):
    from paper_2506_07430_gb300 import moments_batch
    mols = [(8, 4, 4), (6, 3, 2), (10, 5, 5)]
    ks, psis, ab, ints = _batch(torch, "fp64", mols, seed0=2506320)
    N = 96
    got = moments_batch(ks, psis, 0b010, [x[0] for x in ab], [x[1] for x in ab], N)
    n, na, nb = mols[1]
    sc = oracle.SlaterCondon(ints[1].h1, ints[1].eri, n, na, nb)
    psi = psis[1].cpu().numpy()
    ref = okpm.moments_recursion(sc.sigma, sc.dipole(ints[1].dipole[1], psi), ab[1][0], ab[1][1], N)
    assert np.abs(got[1, 0] - ref).max() < 1e-10 * ref[0]
    for k in ks:
        k.close()


def test_batch_state_is_reusable(torch):
    """Single-context calls after a batch and a batch after single-context calls
    give the same moments (reduction counters re-armed, vectors and step counter
    consistent)."""
    from paper_2506_07430_gb300 import moments_batch
    ks, psis, ab, _ = _batch(torch, "fp64", [(6, 3, 3), (8, 4, 4)], seed0=2506340)
    a = [x[0] for x in ab]
    b = [x[1] for x in ab]
    moments_batch(ks, psis, 0b001, a, b, 20)
    ref = ks[1].moments(psis[1], 0b001, a[1], b[1], 20)
    ks[0].recursion_begin(psis[0], 0b001, a[0], b[0], 40)
    ks[0].recursion_advance(9)
    mid = ks[0].recursion_moments()
    got = moments_batch(ks, psis, 0b001, a, b, 20)
    assert np.array_equal(got[0], mid)
    assert np.array_equal(got[1], ref)
    for k in ks:
        k.close()


def test_batch_rejects_bad_lists(torch):
    from paper_2506_07430_gb300 import KPM, KPMError, moments_batch
    ks, psis, ab, ints = _batch(torch, "fp64", [(6, 3, 3), (8, 4, 4)], seed0=2506360)
    a = [x[0] for x in ab]
    b = [x[1] for x in ab]
    with pytest.raises(KPMError, match="KPM_EINVAL"):
        moments_batch([ks[0], ks[0]], [psis[0], psis[0]], 1, a[:1] * 2, b[:1] * 2, 8)
    I = ints[0]
    k32 = KPM(I.h1, I.eri, I.dipole, 6, 3, 3, precision="fp32")
    with pytest.raises(KPMError, match="KPM_EINVAL"):
        moments_batch([ks[0], k32], [psis[0], psis[0]], 1, [a[0]] * 2, [b[0]] * 2, 8)
    kmx = KPM(I.h1, I.eri, I.dipole, 6, 3, 3, precision="mixed")
    with pytest.raises(KPMError, match="KPM_EINVAL"):
        moments_batch([kmx], [psis[0]], 1, [a[0]], [b[0]], 8)
    with pytest.raises(KPMError, match="KPM_EINVAL"):
        moments_batch(ks, psis, 1, a, b, 7)
    # a rescaling that does not contain the spectrum is reported, moments still written
    with pytest.raises(KPMError, match="KPM_EBOUNDS"):
        moments_batch(ks, psis, 1, [a[0], a[1] * 0.2], b, 40)
    out = moments_batch(ks, psis, 1, [a[0], a[1] * 0.2], b, 40, check_bounds=False)
    assert np.array_equal(out[0], ks[0].moments(psis[0], 1, a[0], b[0], 40))
    for k in ks + [k32, kmx]:
        k.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_advance_batch_at_different_steps(torch, prec):
    """Resumable recursions at different steps, advanced together in chunks (with
    single-context advances in between), equal the same recursions advanced alone."""
    from paper_2506_07430_gb300 import recursion_advance_batch
    mols = [(6, 3, 3), (8, 4, 4), (7, 2, 4)]
    ks, psis, ab, _ = _batch(torch, prec, mols, seed0=2506380)
    N = 80
    ref = [k.moments(p, 0b101, a, b, N) for k, p, (a, b) in zip(ks, psis, ab)]
    for k, p, (a, b) in zip(ks, psis, ab):
        k.recursion_begin(p, 0b101, a, b, N)
    ks[1].recursion_advance(3)
    ks[2].recursion_advance(6)
    recursion_advance_batch(ks, 7)              # steps 1..7, 4..10, 7..13
    ks[0].recursion_advance(5)                  # single (graph) steps after a batch
    recursion_advance_batch(ks[1:], 20)
    for k in ks:                                # the rest alone: 27, 9 and 6 steps
        done = k.recursion_moments().shape[1] // 2
        k.recursion_advance(N // 2 - done)
    for i, k in enumerate(ks):
        got = k.recursion_moments()
        assert got.shape == (2, N)
        assert np.array_equal(got, ref[i]), (i, np.abs(got - ref[i]).max())
    for k in ks:
        k.close()
