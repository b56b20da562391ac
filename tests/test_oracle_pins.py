"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: the
Jordan-Wigner Fock-space Hamiltonian built from the operator definition,
closed forms, special cases, exact eigenpairs, or identities of Chebyshev
polynomials.  A dropped term, a wrong sign or index, or a transposed integral
in the oracle makes at least one of them fail (see test_planted_* at the end).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synthetic
from oracle import fock, kpm, strings

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ---------------------------------------------------------------- generator

def test_generator_digests_match_golden():
    with open(os.path.join(GOLDEN, "generator_sha256.json")) as f:
        gold = json.load(f)
    for name, w in synthetic.WORKLOADS.items():
        if w["norb"] > 16:
            continue  # 18-orbital eri is 105 MB; digest still stored, checked on demand
        I = synthetic.integrals(w["norb"], w["nalpha"], w["nbeta"], w["seed"])
        assert synthetic.array_digest(I.h1) == gold[name]["h1"]
        assert synthetic.array_digest(I.eri) == gold[name]["eri"]
        assert synthetic.array_digest(I.dipole) == gold[name]["dipole"]


@pytest.mark.parametrize("n", [4, 8, 12])
def test_eri_eightfold_symmetric_and_psd(n):
    I = synthetic.integrals(n, n // 2, n // 2, seed=100 + n)
    e = I.eri
    for perm in ["qprs", "pqsr", "rspq", "qpsr", "srqp"]:
        assert np.abs(e - np.einsum("pqrs->" + perm, e)).max() < 1e-14
    w = np.linalg.eigvalsh(e.reshape(n * n, n * n))
    assert w.min() > -1e-12
    assert np.abs(I.h1 - I.h1.T).max() == 0.0
    assert np.allclose(np.diag(I.h1), np.linspace(-2, 1, n))
    for c in range(3):
        assert np.abs(I.dipole[c] - I.dipole[c].T).max() == 0.0


# ---------------------------------------------------------------- strings, tables

@pytest.mark.parametrize("n,m", [(4, 2), (6, 3), (8, 4), (9, 2), (10, 5), (12, 6), (5, 0), (5, 5)])
def test_strings_count_and_colex_rank(n, m):
    masks = strings.enumerate_strings(n, m)
    assert len(masks) == math.comb(n, m)
    assert np.all(np.diff(masks) > 0)
    # ascending integer order == combinatorial number system: rank = sum_k C(p_k, k+1)
    for r, x in enumerate(masks.tolist()):
        occ = [p for p in range(n) if (x >> p) & 1]
        assert sum(math.comb(p, k + 1) for k, p in enumerate(occ)) == r


@pytest.mark.parametrize("n,m", [(4, 2), (6, 3), (8, 4), (7, 1), (7, 6)])
def test_table_structure(n, m):
    masks, tgt, pq, sgn = strings.excitation_table(n, m)
    assert tgt.shape == (math.comb(n, m), m * (n - m + 1))
    lut = {int(x): i for i, x in enumerate(masks)}
    for i in range(len(masks)):
        seen = set()
        for k in range(tgt.shape[1]):
            p, q = divmod(int(pq[i, k]), n)
            assert (p, q) not in seen
            seen.add((p, q))
            assert sgn[i, k] in (-1, 1)
            if p == q:
                assert tgt[i, k] == i and sgn[i, k] == 1
            else:
                # E_qp undoes E_pq with the same sign (sign^2 = 1 round trip)
                j = tgt[i, k]
                back = [kk for kk in range(tgt.shape[1]) if pq[j, kk] == q * n + p]
                assert len(back) == 1 and tgt[j, back[0]] == i and sgn[j, back[0]] == sgn[i, k]
                # target string = I - q + p
                assert int(masks[j]) == (int(masks[i]) & ~(1 << q)) | (1 << p)
                # sign = (-1)^(occupied strictly between p and q)
                lo, hi = min(p, q), max(p, q)
                between = int(masks[i]) & (((1 << hi) - 1) & ~((1 << (lo + 1)) - 1))
                assert sgn[i, k] == (-1 if bin(between).count("1") % 2 else 1)
        assert lut[int(masks[i])] == i


def test_table_digests_match_golden():
    with open(os.path.join(GOLDEN, "tables_sha256.json")) as f:
        gold = json.load(f)
    for key in ["8_4", "10_5"]:
        n, m = map(int, key.split("_"))
        masks, tgt, pq, sgn = strings.excitation_table(n, m)
        assert synthetic.array_digest(tgt) == gold[key]["tgt"]
        assert synthetic.array_digest(pq) == gold[key]["pq"]
        assert synthetic.array_digest(sgn) == gold[key]["sgn"]


# ---------------------------------------------------------------- Slater-Condon vs Fock space

SECTORS = [(2, 1, 1), (2, 1, 0), (3, 2, 1), (3, 1, 2), (3, 2, 2), (4, 2, 2), (4, 3, 1), (4, 1, 3)]


@pytest.mark.parametrize("n,na,nb", SECTORS)
def test_slater_condon_equals_jordan_wigner_block(n, na, nb):
    I = synthetic.integrals(n, na, nb, seed=7 + 10 * n + na)
    sc = oracle.SlaterCondon(I.h1, I.eri, n, na, nb)
    H = sc.dense()
    HF = fock.hamiltonian(I.h1, I.eri)
    idx, sg = fock.sector_map(n, sc.masks_a, sc.masks_b)
    block = HF[np.ix_(idx, idx)] * np.outer(sg, sg)
    assert np.abs(block - H).max() < 1e-12
    assert np.abs(H - H.T).max() < 1e-13
    # sector eigenvalues of the full Fock H contain the SC eigenvalues
    w_sc = np.linalg.eigvalsh(H)
    w_bl = np.linalg.eigvalsh(HF[np.ix_(idx, idx)])
    assert np.abs(w_sc - w_bl).max() < 1e-12


@pytest.mark.parametrize("n", [2, 3])
def test_fock_hamiltonian_conserves_n_and_sz(n):
    I = synthetic.integrals(n, 1, 1, seed=3 + n)
    HF = fock.hamiltonian(I.h1, I.eri)
    N, Sz = fock.number_ops(n)
    assert np.abs(HF - HF.T).max() < 1e-13
    assert np.abs(HF @ N - N @ HF).max() < 1e-12
    assert np.abs(HF @ Sz - Sz @ HF).max() < 1e-12


def test_one_electron_hamiltonian_is_h():
    n = 6
    I = synthetic.integrals(n, 1, 0, seed=21)
    sc = oracle.SlaterCondon(I.h1, I.eri, n, 1, 0)
    assert np.abs(sc.dense() - I.h1).max() < 1e-14


def test_no_eri_diagonal_h_gives_orbital_energy_sums():
    n, na, nb = 6, 3, 2
    eps = np.array([-1.3, -0.7, -0.2, 0.4, 0.9, 1.6])
    h1 = np.diag(eps)
    eri = np.zeros((n, n, n, n))
    sc = oracle.SlaterCondon(h1, eri, n, na, nb)
    H = sc.dense()
    assert np.abs(H - np.diag(np.diag(H))).max() == 0.0
    d = []
    for Ia in sc.masks_a:
        for Ib in sc.masks_b:
            d.append(sum(eps[p] for p in range(n) if (Ia >> p) & 1)
                     + sum(eps[p] for p in range(n) if (Ib >> p) & 1))
    assert np.abs(np.diag(H) - np.array(d)).max() < 1e-14


def test_two_orbital_one_alpha_one_beta_closed_form():
    I = synthetic.integrals(2, 1, 1, seed=99)
    h, e = I.h1, I.eri
    sc = oracle.SlaterCondon(h, e, 2, 1, 1)
    H = sc.dense()
    ref = np.zeros((4, 4))
    dets = [(a, b) for a in range(2) for b in range(2)]   # index a*2+b
    for i, (a, b) in enumerate(dets):
        for j, (a2, b2) in enumerate(dets):
            if (a, b) == (a2, b2):
                ref[i, j] = h[a, a] + h[b, b] + e[a, a, b, b]
            elif b == b2:
                ref[i, j] = h[a, a2] + e[a, a2, b, b]
            elif a == a2:
                ref[i, j] = h[b, b2] + e[a, a, b, b2]
            else:
                ref[i, j] = e[a, a2, b, b2]
    assert np.abs(H - ref).max() < 1e-14


def test_trace_closed_form():
    n, na, nb = 6, 3, 2
    I = synthetic.integrals(n, na, nb, seed=12)
    h, e = I.h1, I.eri
    sc = oracle.SlaterCondon(h, e, n, na, nb)
    tr = np.trace(sc.dense())
    Na, Nb = math.comb(n, na), math.comb(n, nb)
    oa, ob = math.comb(n - 1, na - 1), math.comb(n - 1, nb - 1)          # strings containing p
    ta, tb = math.comb(n - 2, na - 2), math.comb(n - 2, nb - 2)          # containing p != q
    ref = sum(h[p, p] for p in range(n)) * (oa * Nb + Na * ob)
    for p in range(n):
        for q in range(n):
            if p != q:
                same = 0.5 * (e[p, p, q, q] - e[p, q, q, p])
                ref += same * (ta * Nb + Na * tb)
            ref += e[p, p, q, q] * oa * ob                                 # alpha-beta Coulomb
    assert abs(tr - ref) < 1e-10 * max(1.0, abs(ref))


def test_dipole_equals_jordan_wigner_one_body():
    n, na, nb = 4, 2, 1
    I = synthetic.integrals(n, na, nb, seed=31)
    sc = oracle.SlaterCondon(I.h1, I.eri, n, na, nb)
    a = fock.annihilators(2 * n)
    d = I.dipole[1]
    mu = sum(-d[p, q] * (a[fock.mode(p, s)].T @ a[fock.mode(q, s)]) for s in range(2)
             for p in range(n) for q in range(n)).toarray()
    idx, sg = fock.sector_map(n, sc.masks_a, sc.masks_b)
    block = mu[np.ix_(idx, idx)] * np.outer(sg, sg)
    x = np.random.default_rng(0).standard_normal(sc.dim)
    assert np.abs(sc.dipole(d, x) - block @ x).max() < 1e-13
    op = oracle.OperatorForm(I.h1, I.eri, n, na, nb)
    assert np.abs(op.dipole(d, x) - block @ x).max() < 1e-13


@pytest.mark.parametrize("n,na,nb", [(4, 2, 2), (5, 3, 2), (6, 3, 3), (6, 2, 4)])
def test_operator_form_equals_slater_condon(n, na, nb):
    I = synthetic.integrals(n, na, nb, seed=50 + n)
    sc = oracle.SlaterCondon(I.h1, I.eri, n, na, nb)
    op = oracle.OperatorForm(I.h1, I.eri, n, na, nb)
    H = sc.dense()
    for j in range(0, sc.dim, max(1, sc.dim // 7)):
        e = np.zeros(sc.dim)
        e[j] = 1.0
        assert np.abs(op.sigma(e) - H[:, j]).max() < 1e-13


def test_operator_form_equals_slater_condon_8o():
    w = synthetic.workload("fci8o8e")
    I = synthetic.integrals(8, 4, 4, w["seed"])
    sc = oracle.SlaterCondon(I.h1, I.eri, 8, 4, 4)
    op = oracle.OperatorForm(I.h1, I.eri, 8, 4, 4)
    x = synthetic.random_state(sc.dim, 1)
    assert np.abs(op.sigma(x) - sc.sigma(x)).max() < 1e-12
    rows = np.arange(0, sc.dim, 37)
    assert np.abs(sc.sigma_rows(rows, x) - sc.csr()[rows] @ x).max() < 1e-12


def test_hash_vector_row_pull_equals_dense_row_pull():
    from oracle.hamiltonian import _lib, hash_vector
    I = synthetic.integrals(8, 4, 4, seed=3)
    sc = oracle.SlaterCondon(I.h1, I.eri, 8, 4, 4)
    x = hash_vector(np.arange(sc.dim))
    assert np.all(np.abs(x) <= 2.0 ** -9) and len(np.unique(x)) > 1000
    assert np.array_equal(x.astype(np.float32).astype(np.float64), x)
    for i in (0, 1, 12345, 2**31 + 7, 2**40 + 3):
        assert _lib().sc_hashvec(i) == hash_vector([i])[0]
    rows = np.arange(0, sc.dim, 13)
    assert np.abs(sc.sigma_rows_hash(rows) - sc.sigma_rows(rows, x)).max() < 1e-15


# ---------------------------------------------------------------- KPM

@pytest.mark.parametrize("N", [2, 16, 256, 2048])
def test_jackson_kernel(N):
    g = kpm.jackson(N)
    assert abs(g[0] - 1.0) < 1e-14
    assert np.all(g > 0) and np.all(g <= 1.0 + 1e-14)
    assert np.all(np.diff(g) < 1e-15)


def test_jackson_damped_delta_is_nonnegative_and_normalised():
    N, M = 128, 1024
    for x0 in (-0.93, -0.2, 0.0, 0.51, 0.97):
        mu = np.cos(np.arange(N) * np.arccos(x0))
        om, dens = kpm.spectrum(mu, 1.0, 0.0, M)
        assert dens.min() > -1e-12 * dens.max()
        # Gauss-Chebyshev: (pi/M) sum_k sin(theta_k) I(x_k) = g_0 Omega_0 = 1
        th = np.arccos(om)
        assert abs(np.pi / M * np.sum(np.sin(th) * dens) - 1.0) < 1e-12
        # peak sits at x0 within the kernel resolution pi/N
        assert abs(om[np.argmax(dens)] - x0) < np.pi / N


def _system8():
    w = synthetic.workload("fci8o8e")
    I = synthetic.integrals(8, 4, 4, w["seed"])
    sc = oracle.SlaterCondon(I.h1, I.eri, 8, 4, 4)
    H = sc.dense()
    E, U = np.linalg.eigh(H)
    return I, sc, H, E, U


def test_ground_state_residual_and_gap():
    I, sc, H, E, U = _system8()
    e0, v0 = oracle.ground_state(sc.sigma, sc.dim)
    assert abs(e0 - E[0]) < 1e-10
    assert np.linalg.norm(H @ v0 - e0 * v0) < 1e-10
    assert E[1] - E[0] > 1e-8


def test_moments_recursion_equals_eigenpairs_8o():
    I, sc, H, E, U = _system8()
    psi0 = U[:, 0]
    a, b = kpm.scale_from_bounds(E[0], E[-1])
    N = 256
    for c in range(3):
        al = sc.dipole(I.dipole[c], psi0)
        w = (U.T @ al) ** 2
        mu_eig = kpm.moments_eigen(E, w, a, b, N)
        mu_rec, direct = kpm.moments_recursion(sc.sigma, al, a, b, N, return_direct=True)
        om0 = al @ al
        assert abs(mu_rec[0] - om0) < 1e-14 * om0                    # sum rule <0|mu^2|0>
        assert np.abs(mu_rec - mu_eig).max() < 1e-10 * om0
        assert np.abs(mu_rec[: len(direct)] - direct).max() < 1e-10 * om0   # doubling == direct
        assert np.all(np.abs(mu_rec) <= om0 * (1 + 1e-12))
        md = kpm.moments_direct(sc.sigma, al, a, b, 64)
        assert np.abs(md - mu_rec[:64]).max() < 1e-11 * om0


def test_spectrum_equals_eigenpair_sum_8o():
    I, sc, H, E, U = _system8()
    psi0 = U[:, 0]
    a, b = kpm.scale_from_bounds(E[0], E[-1])
    N, M = 256, 2048
    al = sc.dipole(I.dipole[2], psi0)
    w = (U.T @ al) ** 2
    mu = kpm.moments_recursion(sc.sigma, al, a, b, N)
    om, dens = kpm.spectrum(mu, a, b, M)
    om2, dens2 = kpm.spectrum_eigen(E, w, a, b, N, M)
    assert np.abs(om - om2).max() < 1e-12
    assert np.linalg.norm(dens - dens2) / np.linalg.norm(dens2) < 1e-10
    # discrete sum rule, energy units: (pi/M) a sum_k sin(theta_k) I_w(w_k) = Omega_0
    th = np.arccos((om - b) / a)
    assert abs(np.pi / M * a * np.sum(np.sin(th) * dens) - mu[0]) < 1e-12 * mu[0]
    assert om[0] < om[-1]


def test_moments_closed_form_without_two_body():
    """ERI = 0, diagonal h: |0> is the aufbau determinant and mu|0> has weight
    (sum_occ 2 d_ii)^2 at E_0 and 2 d_ai^2 at E_0 + e_a - e_i (two spins)."""
    n, m = 6, 3
    eps = np.array([-1.1, -0.6, -0.25, 0.3, 0.8, 1.7])
    h1 = np.diag(eps)
    eri = np.zeros((n, n, n, n))
    d = synthetic.integrals(n, m, m, seed=4).dipole[0]
    sc = oracle.SlaterCondon(h1, eri, n, m, m)
    H = sc.dense()
    E = np.linalg.eigvalsh(H)
    e0 = 2 * eps[:m].sum()
    assert abs(E[0] - e0) < 1e-13
    psi0 = np.zeros(sc.dim)
    psi0[0] = 1.0                       # rank 0 = lowest orbitals occupied, both spins
    al = sc.dipole(d, psi0)
    a, b = kpm.scale_from_bounds(E[0], E[-1])
    N = 64
    mu = kpm.moments_recursion(sc.sigma, al, a, b, N)
    ens = [e0]
    ws = [(2 * np.trace(d[:m, :m])) ** 2]
    for i in range(m):
        for aa in range(m, n):
            ens.append(e0 + eps[aa] - eps[i])
            ws.append(2 * d[aa, i] ** 2)
    ref = kpm.moments_eigen(np.array(ens), np.array(ws), a, b, N)
    assert np.abs(mu - ref).max() < 1e-12 * ref[0]


def test_spectral_bounds_contain_dense_spectrum_8o():
    """ARPACK bounds widened by their Ritz residuals against LAPACK's dense
    eigenvalues (a different routine): they contain the spectrum and are tight."""
    I, sc, H, E, U = _system8()
    lo, hi = oracle.spectral_bounds(sc.sigma, sc.dim)
    width = E[-1] - E[0]
    assert lo <= E[0] and hi >= E[-1], (lo, hi, E[0], E[-1])
    assert E[0] - lo < 1e-8 * width and hi - E[-1] < 1e-8 * width


def test_spectral_bounds_10o_against_plain_lanczos_residuals():
    """10 orbitals (FCI dim 63,504): the extreme Ritz pairs of a plain Lanczos
    iteration with full reorthogonalisation written here (independent of ARPACK's
    implicitly restarted one), with residuals recomputed by the Slater-Condon
    row-pull, lie within the bounds and within their residual of them (an
    eigenvalue lies within |r| of a Ritz value theta)."""
    import scipy.linalg as sl
    I = synthetic.integrals(10, 5, 5, 2506100)
    sc = oracle.SlaterCondon(I.h1, I.eri, 10, 5, 5)
    H = sc.csr()
    lo, hi = oracle.spectral_bounds(sc.sigma, sc.dim)
    k = 160
    Q = np.zeros((k + 1, sc.dim))
    al, be = np.zeros(k), np.zeros(k)
    q = np.random.default_rng(3).standard_normal(sc.dim)
    Q[0] = q / np.linalg.norm(q)
    for j in range(k):
        w = H @ Q[j]
        al[j] = Q[j] @ w
        w -= Q[: j + 1].T @ (Q[: j + 1] @ w)            # full reorthogonalisation, twice
        w -= Q[: j + 1].T @ (Q[: j + 1] @ w)
        be[j] = np.linalg.norm(w)
        Q[j + 1] = w / be[j]
    th, S = sl.eigh_tridiagonal(al, be[:-1])
    for idx, bound, sgn in ((0, lo, 1.0), (k - 1, hi, -1.0)):
        x = Q[:k].T @ S[:, idx]
        x /= np.linalg.norm(x)
        r = np.linalg.norm(sc.sigma(x) - th[idx] * x)      # row-pull, not the CSR
        assert r < 1e-6, r
        assert sgn * (th[idx] + sgn * r - bound) >= 0.0, (bound, th[idx], r)
        assert abs(th[idx] - bound) < 1e-6 * (hi - lo), (bound, th[idx])


def test_block_recursion_equals_column_recursion():
    """moments_recursion_block runs the column recursion on every column of a block
    (H rows generated once per block by the row-pull)."""
    I, sc, H, E, U = _system8()
    a, b = kpm.scale_from_bounds(E[0], E[-1])
    A0 = np.stack([sc.dipole(I.dipole[c], U[:, 0]) for c in range(3)])
    Y = sc.sigma_block(A0)
    for c in range(3):
        assert np.array_equal(Y[c], sc.sigma(A0[c]))
    mb = kpm.moments_recursion_block(sc.sigma_block, A0, a, b, 128)
    for c in range(3):
        mc = kpm.moments_recursion(sc.sigma, A0[c], a, b, 128)
        assert np.abs(mb[c] - mc).max() < 1e-13 * mc[0]


def test_lorentz_kernel_closed_form_and_sum_rule():
    """Lorentz factors: g_0 = 1, strictly decreasing, g_{N-1} = sinh(lam/N)/sinh(lam);
    its spectrum keeps the discrete sum rule and is non-negative for a delta."""
    N, M, lam = 256, 1024, 4.0
    g = kpm.lorentz(N, lam)
    assert g[0] == 1.0 and np.all(np.diff(g) < 0) and g[-1] > 0
    assert abs(g[-1] - np.sinh(lam / N) / np.sinh(lam)) < 1e-15
    for x0 in (-0.9, 0.0, 0.73):
        mu = np.cos(np.arange(N) * np.arccos(x0))
        om, dens = kpm.spectrum(mu, 1.0, 0.0, M, kernel="lorentz", lam=lam)
        th = np.arccos(om)
        assert abs(np.pi / M * np.sum(np.sin(th) * dens) - 1.0) < 1e-12
        assert dens.min() > -1e-12 * dens.max()
        assert abs(om[np.argmax(dens)] - x0) < 2 * np.pi / N


def test_cross_moments_eigenpairs_and_autocorrelation_8o():
    """C_AB moments <0|A T_n B|0> (direct recursion) against the eigenpair sum, and
    A = B against the doubling-identity autocorrelation moments."""
    I, sc, H, E, U = _system8()
    a, b = kpm.scale_from_bounds(E[0], E[-1])
    psi0 = U[:, 0]
    left = -sc.dipole(-I.dipole[0], psi0)        # A|0> with A = sum op E_pq, op = -d^x
    right = -sc.dipole(-I.dipole[1], psi0)       # B|0>, op = -d^y
    mc = kpm.moments_cross(sc.sigma, left, right, a, b, 128)
    me = kpm.moments_cross_eigen(E, U, left, right, a, b, 128)
    assert np.abs(mc - me).max() < 1e-11 * np.sqrt((left @ left) * (right @ right))
    ma = kpm.moments_cross(sc.sigma, left, left, a, b, 128)
    assert np.abs(ma - kpm.moments_recursion(sc.sigma, left, a, b, 128)).max() < 1e-11 * (left @ left)


# ---------------------------------------------------------------- planted mistakes

def test_planted_transposed_eri_is_caught():
    n, na, nb = 3, 2, 1
    I = synthetic.integrals(n, na, nb, seed=77)
    HF = fock.hamiltonian(I.h1, I.eri)
    bad = np.einsum("pqrs->prqs", I.eri)       # physicist/chemist mix-up
    sc = oracle.SlaterCondon(I.h1, bad, n, na, nb)
    idx, sg = fock.sector_map(n, sc.masks_a, sc.masks_b)
    assert np.abs(HF[np.ix_(idx, idx)] * np.outer(sg, sg) - sc.dense()).max() > 1e-3


def test_planted_jackson_typo_is_caught():
    N = 64
    n = np.arange(N)
    q = np.pi / (N + 1)
    printed = ((N - n - 1) * np.cos(q * n) + np.sin(q * n) / np.tan(q)) / (N + 1)
    assert abs(printed[0] - 1.0) > 1e-3      # the g_0 = 1 pin rejects the printed factor


def test_planted_doubling_sign_is_caught():
    I, sc, H, E, U = _system8()
    a, b = kpm.scale_from_bounds(E[0], E[-1])
    al = sc.dipole(I.dipole[0], U[:, 0])
    mu = kpm.moments_recursion(sc.sigma, al, a, b, 16)
    w = (U.T @ al) ** 2
    ref = kpm.moments_eigen(E, w, a, b, 16)
    bad = mu.copy()
    bad[3::2] = bad[3::2] + 2 * mu[1]        # Omega_2n+1 = 2t_n + Omega_1 instead of - Omega_1
    assert np.abs(bad - ref).max() > 1e-6 * ref[0]
    assert np.abs(mu - ref).max() < 1e-10 * ref[0]
