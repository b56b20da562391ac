"""Parity of the CUDA path (through the C-ABI) with the CPU FP64 oracle.

Tolerances:
* string tables: bit-exact;
* FP64 sigma: |dy| <= 1e-12 * max|y| (FP64 rounding of sums of ~1e3-1e4 terms);
* FP32 sigma: |dy| <= 2e-6 * max|y| (FP32 unit roundoff 6e-8 times the growth of
  sums of ~1e3 terms, with headroom);
* moments: FP64 <= 1e-10 Omega_0.  For paths with FP32 vectors the error grows
  linearly with the moment index (a systematic eigenvalue shift dE moves
  Omega_n by ~ n dE / a): bound 4 N u Omega_0 with u the relative error per
  H-element product of the path (FP32 2^-24, split FP16 2^-22, split BF16 2^-16);
  measured values are printed by the tests;
* spectrum: relative L2 <= 1e-10 for identical moments (FP64 sums on both sides).
"""
import math

import numpy as np
import pytest

import oracle
import synthetic
from oracle import kpm as okpm
from oracle import strings as ostr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available()
    return _t


def _kpm(I, n, na, nb, prec):
    from paper_2506_07430_gb300 import KPM
    return KPM(I.h1, I.eri, I.dipole, n, na, nb, precision=prec)


# ---------------------------------------------------------------- tables

@pytest.mark.parametrize("n,na,nb", [(8, 4, 4), (10, 5, 5), (12, 6, 6), (14, 7, 7), (16, 8, 8),
                                     (7, 2, 5), (5, 5, 0), (1, 1, 0), (9, 1, 8)])
def test_string_tables_bit_exact(torch, n, na, nb):
    I = synthetic.integrals(n, na, nb, seed=1000 + n)
    k = _kpm(I, n, na, nb, "fp64")
    for spin, m in ((0, na), (1, nb)):
        masks, tgt, pq, sgn = ostr.excitation_table(n, m)
        gm, gt, gp, gs = k.string_table(spin)
        assert np.array_equal(gm.astype(np.int64), masks)
        assert np.array_equal(gt, tgt)
        assert np.array_equal(gp, pq)
        assert np.array_equal(gs, sgn)
    assert k.dim == math.comb(n, na) * math.comb(n, nb)
    k.close()


def test_string_tables_18_orbitals_sampled(torch):
    n, m = 18, 9
    I = synthetic.integrals(n, m, m, seed=2506075)
    k = _kpm(I, n, m, m, "fp32")
    gm, gt, gp, gs = k.string_table(0)
    masks = ostr.enumerate_strings(n, m)
    assert np.array_equal(gm.astype(np.int64), masks)
    lut = ostr.rank_lookup(n, masks)
    rows = np.random.default_rng(5).choice(len(masks), 400, replace=False)
    for r in rows:
        I0 = int(masks[r])
        kk = 0
        for q in range(n):
            if not (I0 >> q) & 1:
                continue
            for p in sorted([q] + [x for x in range(n) if not (I0 >> x) & 1]):
                m1, s1 = ostr.apply_annihilator(I0, q)
                m2, s2 = ostr.apply_creator(m1, p)
                assert gt[r, kk] == lut[m2] and gp[r, kk] == p * n + q and gs[r, kk] == s1 * s2
                kk += 1
    k.close()


# ---------------------------------------------------------------- sigma, dipole

SMALL = [(8, 4, 4), (6, 3, 2), (7, 2, 4), (5, 5, 0), (5, 0, 3), (4, 1, 1), (1, 1, 1), (10, 5, 5)]


def _sc(n, na, nb, seed):
    I = synthetic.integrals(n, na, nb, seed)
    return I, oracle.SlaterCondon(I.h1, I.eri, n, na, nb)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("n,na,nb", SMALL)
def test_sigma_full(torch, prec, tol, n, na, nb):
    I, sc = _sc(n, na, nb, seed=300 + 7 * n + na)
    k = _kpm(I, n, na, nb, prec)
    X = np.stack([synthetic.random_state(sc.dim, s) for s in (1, 2)])
    ref = np.stack([sc.sigma(x) for x in X])
    xt = torch.tensor(X, dtype=k.vdtype, device="cuda")
    y = k.sigma(xt).cpu().numpy().astype(np.float64)
    if prec == "fp32":
        ref = np.stack([sc.sigma(x.astype(np.float32).astype(np.float64)) for x in X])
    err = np.abs(y - ref).max() / np.abs(ref).max()
    assert err < tol, err
    k.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_sigma_12_orbitals_full(torch, prec, tol):
    n = 12
    w = synthetic.workload("fci12o12e")
    I, sc = _sc(n, 6, 6, seed=w["seed"])
    k = _kpm(I, n, 6, 6, prec)
    x = synthetic.random_state(sc.dim, 3)
    if prec == "fp32":
        x = x.astype(np.float32).astype(np.float64)
    ref = sc.sigma(x)
    y = k.sigma(torch.tensor(x, dtype=k.vdtype, device="cuda")).cpu().numpy()
    assert np.abs(y - ref).max() / np.abs(ref).max() < tol
    k.close()


@pytest.mark.parametrize("n,na,nb,prec,tol", [(14, 7, 7, "fp64", 1e-12), (14, 7, 7, "fp32", 2e-6),
                                              (16, 8, 8, "fp32", 2e-6)])
def test_sigma_sampled_rows(torch, n, na, nb, prec, tol):
    w = {14: 2506150, 16: 2506073}[n]
    I, sc = _sc(n, na, nb, seed=w)
    k = _kpm(I, n, na, nb, prec)
    x = synthetic.random_state(sc.dim, 4)
    if prec == "fp32":
        x = x.astype(np.float32).astype(np.float64)
    y = k.sigma(torch.tensor(x, dtype=k.vdtype, device="cuda")).cpu().numpy()
    rng = np.random.default_rng(9)
    rows = np.concatenate([rng.choice(sc.dim, 4000, replace=False), [0, sc.dim - 1]])
    ref = sc.sigma_rows(rows, x)
    assert np.abs(y[rows] - ref).max() / np.abs(ref).max() < tol
    k.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-7)])
@pytest.mark.parametrize("n,na,nb", [(8, 4, 4), (7, 2, 4), (10, 5, 5)])
def test_dipole(torch, prec, tol, n, na, nb):
    I, sc = _sc(n, na, nb, seed=77 + n)
    k = _kpm(I, n, na, nb, prec)
    psi = synthetic.random_state(sc.dim, 6)
    pt = torch.tensor(psi, dtype=torch.float64, device="cuda")
    for c in range(3):
        ref = sc.dipole(I.dipole[c], psi)
        y = k.apply_dipole(c, pt).cpu().numpy()
        assert np.abs(y - ref).max() / np.abs(ref).max() < tol
    k.close()


# ---------------------------------------------------------------- moments, spectrum

@pytest.fixture(scope="module")
def sys8():
    w = synthetic.workload("fci8o8e")
    I, sc = _sc(8, 4, 4, seed=w["seed"])
    E, U = np.linalg.eigh(sc.dense())
    a, b = okpm.scale_from_bounds(E[0], E[-1])
    return I, sc, E, U, a, b


def _moment_bound(prec, N):
    u = {"fp32": 2.0 ** -24, "mixed": 2.0 ** -22, "mixed_bf16": 2.0 ** -16}[prec]
    return 4 * N * u


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", _moment_bound("fp32", 256))])
def test_moments_8o_ground_state(torch, sys8, prec, tol):
    I, sc, E, U, a, b = sys8
    psi0 = U[:, 0]
    N = 256
    k = _kpm(I, 8, 4, 4, prec)
    mom = k.moments(torch.tensor(psi0, device="cuda"), 0b111, a, b, N)
    for c in range(3):
        al = sc.dipole(I.dipole[c], psi0)
        ref = okpm.moments_eigen(E, (U.T @ al) ** 2, a, b, N)
        print(prec, "8o moment error / Omega_0:", np.abs(mom[c] - ref).max() / ref[0])
        assert np.abs(mom[c] - ref).max() < tol * ref[0], (c, np.abs(mom[c] - ref).max() / ref[0])
    # host-buffer entry point gives the same numbers
    mom_h = k.moments(psi0, 0b101, a, b, N)
    assert np.array_equal(mom_h, mom[[0, 2]])
    k.close()


def test_moments_resumable_equals_one_shot(torch, sys8):
    I, sc, E, U, a, b = sys8
    k = _kpm(I, 8, 4, 4, "fp64")
    psi = torch.tensor(U[:, 0], device="cuda")
    one = k.moments(psi, 0b010, a, b, 64)
    k.recursion_begin(psi, 0b010, a, b, 64)
    parts = []
    for s in (5, 10, 16):
        k.recursion_advance(s)
        parts.append(k.recursion_moments())
    assert parts[-1].shape == (1, 64)
    assert np.array_equal(parts[-1], one)
    assert np.array_equal(parts[0], one[:, :12])
    k.close()


def test_moments_10o_random_state(torch):
    n = 10
    I, sc = _sc(n, 5, 5, seed=2506100)
    sc.csr()
    emin, emax = oracle.spectral_bounds(sc.sigma, sc.dim)
    a, b = okpm.scale_from_bounds(emin, emax)
    psi = synthetic.random_state(sc.dim, 8)
    N = 128
    for prec, tol in (("fp64", 1e-10), ("fp32", 1e-6)):
        k = _kpm(I, n, 5, 5, prec)
        mom = k.moments(torch.tensor(psi, device="cuda"), 0b001, a, b, N)
        ref = okpm.moments_recursion(sc.sigma, sc.dipole(I.dipole[0], psi), a, b, N)
        assert np.abs(mom[0] - ref).max() < tol * ref[0], (prec, np.abs(mom[0] - ref).max() / ref[0])
        k.close()


def test_bounds_contain_spectrum(torch, sys8):
    I, sc, E, U, a, b = sys8
    for prec in ("fp64", "fp32"):
        k = _kpm(I, 8, 4, 4, prec)
        lo, hi = k.bounds(iters=80, seed=3)
        assert lo <= E[0] + 1e-9 and hi >= E[-1] - 1e-9, (lo, hi, E[0], E[-1])
        assert (hi - lo) < 1.05 * (E[-1] - E[0])
        k.close()


def test_ebounds_detected(torch, sys8):
    from paper_2506_07430_gb300 import KPMError
    I, sc, E, U, a, b = sys8
    k = _kpm(I, 8, 4, 4, "fp64")
    with pytest.raises(KPMError, match="KPM_EBOUNDS"):
        k.moments(torch.tensor(U[:, 0], device="cuda"), 1, 0.3 * a, b, 64)
    k.close()


def test_spectrum_matches_oracle(torch, sys8):
    from paper_2506_07430_gb300 import spectrum
    I, sc, E, U, a, b = sys8
    psi0 = U[:, 0]
    N, M = 256, 2048
    mom = sum(okpm.moments_recursion(sc.sigma, sc.dipole(I.dipole[c], psi0), a, b, N)
              for c in range(3))
    for kern in ("jackson", "none"):
        om, it = spectrum(mom, a, b, M, kern)
        om_r, it_r = okpm.spectrum(mom, a, b, M, kern)
        assert np.abs(om - om_r).max() < 1e-13 * (abs(a) + abs(b))
        assert np.linalg.norm(it - it_r) / np.linalg.norm(it_r) < 1e-10
    # Eq. 1 from exact eigenpairs, Jackson-broadened, equals the reconstruction
    w = sum((U.T @ sc.dipole(I.dipole[c], psi0)) ** 2 for c in range(3))
    om_e, it_e = okpm.spectrum_eigen(E, w, a, b, N, M)
    om, it = spectrum(mom, a, b, M)
    assert np.linalg.norm(it - it_e) / np.linalg.norm(it_e) < 1e-9


def test_spectrum_edge_sizes(torch):
    from paper_2506_07430_gb300 import spectrum
    for N, M in ((1, 1), (2, 3), (3000, 257)):
        mu = np.cos(np.arange(N) * 0.7) * 0.5
        om, it = spectrum(mu, 1.3, -0.2, M)
        om_r, it_r = okpm.spectrum(mu, 1.3, -0.2, M)
        assert np.allclose(om, om_r, rtol=0, atol=1e-13)
        assert np.linalg.norm(it - it_r) <= 1e-10 * max(1e-300, np.linalg.norm(it_r))


# ---------------------------------------------------------------- tensor-core (KPM_MIXED)

# Tensor-core variants: "mixed" splits x into 2 and the integrals into 3 FP16
# pieces (4 MMAs, ~22 significant bits per product, like FP32 to a factor ~4);
# "mixed_bf16" splits both into 2 BF16 pieces (3 MMAs, ~16 bits).  Sums of O(100)
# products are compared with these bounds relative to max|y|.
MIXED_TOL = {"mixed": 1e-5, "mixed_bf16": 1e-4}
MIXED = list(MIXED_TOL)


@pytest.mark.parametrize("prec", MIXED)
@pytest.mark.parametrize("n,na,nb", [(8, 4, 4), (6, 3, 2), (7, 2, 4), (5, 5, 0), (5, 0, 3),
                                     (4, 1, 1), (1, 1, 1), (10, 5, 5)])
def test_sigma_mixed_one_body_only(torch, prec, n, na, nb):
    I = synthetic.integrals(n, na, nb, seed=500 + n)
    eri0 = np.zeros_like(I.eri)
    sc = oracle.SlaterCondon(I.h1, eri0, n, na, nb)
    from paper_2506_07430_gb300 import KPM
    k = KPM(I.h1, eri0, I.dipole, n, na, nb, precision=prec)
    x = synthetic.random_state(sc.dim, 11).astype(np.float32).astype(np.float64)
    y = k.sigma(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    k.synchronize()
    ref = sc.sigma(x)
    assert np.abs(y - ref).max() / np.abs(ref).max() < MIXED_TOL[prec]
    k.close()


@pytest.mark.parametrize("prec", MIXED)
@pytest.mark.parametrize("n,na,nb", SMALL + [(12, 6, 6)])
def test_sigma_mixed_full(torch, prec, n, na, nb):
    seed = 300 + 7 * n + na if n != 12 else synthetic.workload("fci12o12e")["seed"]
    I, sc = _sc(n, na, nb, seed=seed)
    k = _kpm(I, n, na, nb, prec)
    X = np.stack([synthetic.random_state(sc.dim, s) for s in (1, 2)]).astype(np.float32)
    y = k.sigma(torch.tensor(X, device="cuda")).cpu().numpy()
    k.synchronize()
    ref = np.stack([sc.sigma(x.astype(np.float64)) for x in X])
    err = np.abs(y - ref).max() / np.abs(ref).max()
    print(prec, (n, na, nb), "sigma error / max|y|:", err)
    assert err < MIXED_TOL[prec], err
    k.close()


@pytest.mark.parametrize("prec", MIXED)
def test_sigma_mixed_fixed_point_range(torch, prec):
    """A state whose values align every term of one opposite-spin sum, so that
    row's fixed-point sum reaches a large part of the a-priori range of the
    scatter (more than a quarter of it): the integer accumulation must neither
    overflow nor lose the small terms elsewhere."""
    n, na, nb, seed = 8, 4, 4, 2506071
    I, sc = _sc(n, na, nb, seed=seed)
    masks, tgt, pq, sgn = ostr.excitation_table(n, na)
    nexc = pq.shape[1]

    def slot(v):
        p, q = divmod(int(v), n)
        return max(p, q) * (max(p, q) + 1) // 2 + min(p, q)

    nsl = n * (n + 1) // 2
    W = np.zeros((nsl, nsl))
    for p in range(n):
        for q in range(n):
            for r in range(n):
                for s in range(n):
                    W[slot(p * n + q), slot(r * n + s)] = I.eri[p, q, r, s]
    R0 = 14
    coef = {}
    for e in range(nexc):
        for f in range(nexc):
            key = (int(tgt[R0, e]), int(tgt[R0, f]))
            coef[key] = coef.get(key, 0.0) + sgn[R0, e] * sgn[R0, f] * W[slot(pq[R0, e]),
                                                                            slot(pq[R0, f])]
    N = len(masks)
    x = 1e-3 * synthetic.random_state(N * N, 11) * math.sqrt(N * N)
    X = x.reshape(N, N)
    for (a, b), c in coef.items():
        X[a, b] = 1.0 if c >= 0 else -1.0
    # the aligned sum against the a-priori bound of the fixed-point scale
    aligned = sum(abs(c) for c in coef.values())
    bound = 1.02 * nexc * 1.0 * np.abs(W).sum(axis=0).max()
    assert aligned > bound / 4, (aligned, bound)
    x = X.reshape(-1).astype(np.float32)
    k = _kpm(I, n, na, nb, prec)
    y = k.sigma(torch.tensor(x[None, :], device="cuda")).cpu().numpy()[0]
    k.synchronize()
    ref = sc.sigma(x.astype(np.float64))
    err = np.abs(y - ref).max() / np.abs(ref).max()
    print(prec, "aligned-sum state: sigma error / max|y|:", err)
    assert err < MIXED_TOL[prec], err
    k.close()


@pytest.mark.parametrize("prec", MIXED)
@pytest.mark.parametrize("n,na,nb", [(14, 7, 7), (16, 8, 8)])
def test_sigma_mixed_sampled_rows(torch, prec, n, na, nb):
    w = {14: 2506150, 16: 2506073}[n]
    I, sc = _sc(n, na, nb, seed=w)
    k = _kpm(I, n, na, nb, prec)
    x = synthetic.random_state(sc.dim, 4).astype(np.float32)
    y = k.sigma(torch.tensor(x, device="cuda")).cpu().numpy()
    k.synchronize()
    rng = np.random.default_rng(9)
    rows = np.concatenate([rng.choice(sc.dim, 4000, replace=False), [0, sc.dim - 1]])
    ref = sc.sigma_rows(rows, x.astype(np.float64))
    err = np.abs(y[rows] - ref).max() / np.abs(ref).max()
    print(prec, n, "sampled sigma error / max|y|:", err)
    assert err < MIXED_TOL[prec]
    k.close()


@pytest.mark.parametrize("prec", MIXED)
def test_moments_mixed_8o(torch, sys8, prec):
    I, sc, E, U, a, b = sys8
    psi0 = U[:, 0]
    N = 256
    k = _kpm(I, 8, 4, 4, prec)
    mom = k.moments(torch.tensor(psi0, device="cuda"), 0b111, a, b, N)
    errs = []
    for c in range(3):
        al = sc.dipole(I.dipole[c], psi0)
        ref = okpm.moments_eigen(E, (U.T @ al) ** 2, a, b, N)
        errs.append(np.abs(mom[c] - ref).max() / ref[0])
    print(prec, "8o moment error / Omega_0:", errs)
    assert max(errs) < _moment_bound(prec, N), errs
    k.close()


def _hash_vector_dev(torch, dim):
    """The oracle's hash test vector built on the device in chunks (exact in FP32)."""
    x = torch.empty(dim, dtype=torch.float32, device="cuda")
    C = 0x9E3779B97F4A7C15 - (1 << 64)          # same bits as a signed int64
    step = 1 << 27
    for s0 in range(0, dim, step):
        i = torch.arange(s0, min(dim, s0 + step), device="cuda", dtype=torch.int64)
        h = ((i * C) >> 48) & 0xFFFF            # wrap-around multiply, low 16 bits of the shift
        x[s0:s0 + len(i)] = ((h - 32768).to(torch.float64) / 16777216.0).to(torch.float32)
    return x


def test_sigma_18_orbitals_sampled_rows(torch):
    """18 orbitals, 9+9 electrons (FCI dim 2,363,904,400, int64 indexing): FP32 sigma
    on sampled rows vs the oracle's Slater-Condon row-pull."""
    from oracle.hamiltonian import hash_vector
    n, m = 18, 9
    I = synthetic.integrals(n, m, m, seed=2506075)
    k = _kpm(I, n, m, m, "fp32")
    dim = k.dim
    assert dim == math.comb(18, 9) ** 2 and dim > 2**31
    x = _hash_vector_dev(torch, dim)
    probe = np.array([0, 1, 2**31 + 5, dim - 1])
    assert np.array_equal(x[torch.tensor(probe, device="cuda")].cpu().numpy().astype(np.float64),
                          hash_vector(probe))
    y = k.sigma(x)
    k.synchronize()
    del x
    sc = oracle.SlaterCondon(I.h1, I.eri, n, m, m)
    rng = np.random.default_rng(18)
    rows = np.concatenate([rng.choice(dim, 3000, replace=False), [0, dim - 1, 2**31 + 5]])
    ref = sc.sigma_rows_hash(rows)
    got = y[torch.tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 2e-6
    k.close()


@pytest.mark.parametrize("prec,n,ne", [("fp64", 8, 4), ("fp32", 10, 5), ("mixed", 10, 5)])
def test_graph_steps_equal_direct_steps(torch, prec, n, ne):
    """Recursion steps replayed from captured CUDA graphs give the same moments,
    bit for bit, as the same steps issued kernel by kernel (chunk sizes mix graph
    replays and single steps, and both vector assignments)."""
    I = synthetic.integrals(n, ne, ne, 2506200 + n)
    out = []
    for graphs in (True, False):
        k = _kpm(I, n, ne, ne, prec)
        k.graphs_enable(graphs)
        psi = torch.from_numpy(synthetic.random_state(k.dim, 5)).cuda()
        emin, emax = k.bounds(iters=40, seed=3)
        a, b = k.scale(emin, emax)
        k.recursion_begin(psi, 0b101, a, b, 2 * 40)
        for chunk in (3, 2, 7, 1, 6, 4, 5, 11):
            k.recursion_advance(chunk)
        out.append(k.recursion_moments())
        k.close()
    assert out[0].shape == (2, 80)
    assert np.array_equal(out[0], out[1])


def test_autotuned_gemm_groups(torch):
    """The autotuner's rasterisation choices are among its candidates (14 orbitals
    and up are tuned, smaller shapes keep 16), and tuning leaves results alone:
    the tuned context's sigma matches the oracle on sampled rows like any other."""
    I = synthetic.integrals(8, 4, 4, 2506071)
    k = _kpm(I, 8, 4, 4, "mixed")
    assert k.tuned_params() == (16, 16)
    k.close()
    k = _kpm(I, 8, 4, 4, "fp64")
    assert k.tuned_params() == (0, 0)
    k.close()
    I = synthetic.integrals(14, 7, 7, 2506074)
    k = _kpm(I, 14, 7, 7, "mixed")
    gb, ga = k.tuned_params()
    assert gb in (4, 8, 16, 32) and ga in (4, 8, 16, 32)
    k.close()
