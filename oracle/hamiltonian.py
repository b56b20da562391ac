"""FP64 CPU Hamiltonian, dipole and sigma for the determinant basis.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline import this module.  It shares no code with the CUDA library.

Two independent routes to H x:

* ``SlaterCondon`` -- the determinant-pair Slater-Condon matrix of the paper's
  second-quantized Hamiltonian (Methods, "Mapping fermionic Hamiltonians to the
  qubits"), from the C file ``sc.c`` (rows on demand, or the full CSR at small
  sizes).  This is the definition written out.
* ``OperatorForm`` -- the same Hamiltonian applied operator by operator in
  NumPy: H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - d_qr E_ps)
  with E_pq = E^alpha_pq + E^beta_pq, each E applied with the brute-force string
  tables of ``strings.py``; the sum over (r, s) is a matrix product.  It exists
  because the determinant rules are too slow for full vectors at 12 orbitals;
  the tests pin it to ``SlaterCondon`` entry by entry.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

from . import strings as _strings

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``sc.c`` into ``_build/libscoracle.so`` next to this file."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libscoracle.so")
    src = os.path.join(_HERE, "sc.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               src, "-o", tmp])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            so = build()
            lib = ctypes.CDLL(so)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.sc_row_capacity.restype = I64
            lib.sc_row_capacity.argtypes = [P]
            lib.sc_row.restype = I64
            lib.sc_row.argtypes = [P, I64, P, P]
            lib.sc_sigma_rows.restype = None
            lib.sc_sigma_rows.argtypes = [P, P, I64, P, P]
            lib.sc_sigma.restype = None
            lib.sc_sigma.argtypes = [P, P, P]
            lib.sc_sigma_block.restype = None
            lib.sc_sigma_block.argtypes = [P, P, P, ctypes.c_int]
            lib.sc_row_counts.restype = None
            lib.sc_row_counts.argtypes = [P, P]
            lib.sc_fill_csr.restype = None
            lib.sc_fill_csr.argtypes = [P, P, P, P]
            lib.sc_dipole_rows.restype = None
            lib.sc_dipole_rows.argtypes = [P, P, P, I64, P, P]
            lib.sc_omp_threads.restype = ctypes.c_int
            lib.sc_set_threads.restype = None
            lib.sc_set_threads.argtypes = [ctypes.c_int]
            lib.sc_sigma_rows_hash.restype = None
            lib.sc_sigma_rows_hash.argtypes = [P, P, I64, P]
            lib.sc_hashvec.restype = ctypes.c_double
            lib.sc_hashvec.argtypes = [I64]
            _LIB = lib
    return _LIB


def omp_threads() -> int:
    return int(_lib().sc_omp_threads())


def set_omp_threads(n: int) -> None:
    """Threads of the later oracle calls (timing on one core or on all)."""
    _lib().sc_set_threads(int(n))


class _CSys(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("na", ctypes.c_int), ("nb", ctypes.c_int),
                ("nsa", ctypes.c_int64), ("nsb", ctypes.c_int64),
                ("h1", ctypes.c_void_p), ("eri", ctypes.c_void_p),
                ("masks_a", ctypes.c_void_p), ("masks_b", ctypes.c_void_p),
                ("rank_a", ctypes.c_void_p), ("rank_b", ctypes.c_void_p)]


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def hash_vector(idx) -> np.ndarray:
    """x(i) = ((((i * 0x9E3779B97F4A7C15) >> 48) & 0xFFFF) - 32768) * 2^-24, 64-bit
    wrap-around multiply; exactly representable in FP32 and FP64."""
    i = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h = (i * np.uint64(0x9E3779B97F4A7C15)) >> np.uint64(48)
    return ((h & np.uint64(0xFFFF)).astype(np.int64) - 32768).astype(np.float64) / 16777216.0


class SlaterCondon:
    """Determinant-pair Slater-Condon H and the one-body dipole (FP64)."""

    def __init__(self, h1, eri, norb, nalpha, nbeta):
        self.n, self.na, self.nb = int(norb), int(nalpha), int(nbeta)
        self.h1 = np.ascontiguousarray(h1, dtype=np.float64)
        self.eri = np.ascontiguousarray(eri, dtype=np.float64).reshape(-1)
        self.masks_a = _strings.enumerate_strings(norb, nalpha)
        self.masks_b = _strings.enumerate_strings(norb, nbeta)
        self.rank_a = _strings.rank_lookup(norb, self.masks_a)
        self.rank_b = _strings.rank_lookup(norb, self.masks_b)
        self.nsa, self.nsb = len(self.masks_a), len(self.masks_b)
        self.dim = self.nsa * self.nsb
        self._c = _CSys(self.n, self.na, self.nb, self.nsa, self.nsb,
                        _ptr(self.h1), _ptr(self.eri), _ptr(self.masks_a),
                        _ptr(self.masks_b), _ptr(self.rank_a), _ptr(self.rank_b))
        self._csr = None

    def _cp(self):
        return ctypes.addressof(self._c)

    def row(self, r: int):
        """(columns, values) of row r; the diagonal comes first."""
        lib = _lib()
        cap = lib.sc_row_capacity(self._cp())
        cols = np.empty(cap, np.int64)
        vals = np.empty(cap, np.float64)
        k = lib.sc_row(self._cp(), int(r), _ptr(cols), _ptr(vals))
        return cols[:k].copy(), vals[:k].copy()

    def sigma_rows(self, rows, x):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert x.shape == (self.dim,)
        y = np.empty(len(rows), np.float64)
        _lib().sc_sigma_rows(self._cp(), _ptr(rows), len(rows), _ptr(x), _ptr(y))
        return y

    def sigma_rows_hash(self, rows):
        """Rows of H x for the hash test vector x(i) (see ``hash_vector``)."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        y = np.empty(len(rows), np.float64)
        _lib().sc_sigma_rows_hash(self._cp(), _ptr(rows), len(rows), _ptr(y))
        return y

    def sigma(self, x):
        if self._csr is not None:
            return self._csr @ x
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.dim, np.float64)
        _lib().sc_sigma(self._cp(), _ptr(x), _ptr(y))
        return y

    def sigma_block(self, X):
        """Y[c] = H X[c] for a block X of shape (ncol, dim): each row of H is
        generated once for all columns (the same per-column sums as ``sigma``)."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        assert X.ndim == 2 and X.shape[1] == self.dim
        if self._csr is not None:
            return np.ascontiguousarray((self._csr @ X.T).T)
        Y = np.empty_like(X)
        _lib().sc_sigma_block(self._cp(), _ptr(X), _ptr(Y), X.shape[0])
        return Y

    def csr(self) -> sp.csr_matrix:
        """Full sparse H (dims up to a few 1e5 only)."""
        if self._csr is None:
            lib = _lib()
            counts = np.empty(self.dim, np.int64)
            lib.sc_row_counts(self._cp(), _ptr(counts))
            indptr = np.zeros(self.dim + 1, np.int64)
            np.cumsum(counts, out=indptr[1:])
            nnz = int(indptr[-1])
            indices = np.empty(nnz, np.int64)
            data = np.empty(nnz, np.float64)
            lib.sc_fill_csr(self._cp(), _ptr(indptr), _ptr(indices), _ptr(data))
            m = sp.csr_matrix((data, indices, indptr), shape=(self.dim, self.dim))
            m.sum_duplicates()
            self._csr = m
        return self._csr

    def dense(self) -> np.ndarray:
        return self.csr().toarray()

    def dipole_rows(self, d, rows, x):
        d = np.ascontiguousarray(d, dtype=np.float64)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(len(rows), np.float64)
        _lib().sc_dipole_rows(self._cp(), _ptr(d), _ptr(rows), len(rows), _ptr(x), _ptr(y))
        return y

    def dipole(self, d, x):
        return self.dipole_rows(d, np.arange(self.dim, dtype=np.int64), x)


class OperatorForm:
    """H x by applying E_pq operators with the brute-force string tables (NumPy)."""

    def __init__(self, h1, eri, norb, nalpha, nbeta):
        self.n, self.na, self.nb = int(norb), int(nalpha), int(nbeta)
        n = self.n
        self.h1 = np.asarray(h1, np.float64)
        self.eri = np.asarray(eri, np.float64).reshape(n, n, n, n)
        _, self.tgt_a, self.pq_a, self.sgn_a = _strings.excitation_table(n, nalpha)
        if nbeta == nalpha:
            self.tgt_b, self.pq_b, self.sgn_b = self.tgt_a, self.pq_a, self.sgn_a
        else:
            _, self.tgt_b, self.pq_b, self.sgn_b = _strings.excitation_table(n, nbeta)
        self.nsa, self.nsb = self.tgt_a.shape[0], self.tgt_b.shape[0]
        self.dim = self.nsa * self.nsb
        # k_ps = h_ps - 1/2 sum_q (pq|qs): moves the d_qr E_ps term into the one-body part
        self.k = self.h1 - 0.5 * np.einsum("pqqs->ps", self.eri)
        self.V = self.eri.reshape(n * n, n * n)

    def _groups(self, tgt, pq, sgn):
        """Table entries grouped by pair index: for each pq, (J, I, s) with
        a+_p a_q |J> = s |I>.  Within one pq the map J -> I is one-to-one."""
        ns, ne = tgt.shape
        J = np.repeat(np.arange(ns), ne)
        I = tgt.reshape(-1).astype(np.int64)
        P = pq.reshape(-1).astype(np.int64)
        S = sgn.reshape(-1).astype(np.float64)
        out = []
        for g in range(self.n * self.n):
            m = P == g
            out.append((J[m], I[m], S[m]))
        return out

    def apply_E(self, C: np.ndarray) -> np.ndarray:
        """D[pq] = E_pq C for all pq; C shaped (nsa, nsb); returns (n*n, nsa, nsb).

        <I|E_pq|J> is nonzero when a+_p a_q |J> = s |I>, i.e. when J's table
        has the entry (pq -> I, s); so E_pq C places s * C[J] at I.
        """
        if not hasattr(self, "_ga"):
            self._ga = self._groups(self.tgt_a, self.pq_a, self.sgn_a)
            self._gb = self._groups(self.tgt_b, self.pq_b, self.sgn_b)
        n2 = self.n * self.n
        D = np.zeros((n2, self.nsa, self.nsb))
        for g in range(n2):
            J, I, S = self._ga[g]
            D[g, I, :] += S[:, None] * C[J, :]
            J, I, S = self._gb[g]
            D[g][:, I] += S[None, :] * C[:, J]
        return D

    def sigma(self, x: np.ndarray) -> np.ndarray:
        C = np.asarray(x, np.float64).reshape(self.nsa, self.nsb)
        n2 = self.n * self.n
        D = self.apply_E(C)                                    # E_rs C
        G = (self.V @ D.reshape(n2, -1)).reshape(n2, self.nsa, self.nsb)  # sum_rs (pq|rs) E_rs C
        del D
        G *= 0.5
        G += self.k.reshape(n2, 1, 1) * C[None]                # one-body k_pq, applied by the outer E_pq
        out = np.zeros((self.nsa, self.nsb))
        for g in range(n2):                                    # sigma = sum_pq E_pq G[pq]
            J, I, S = self._ga[g]
            out[I, :] += S[:, None] * G[g, J, :]
            J, I, S = self._gb[g]
            out[:, I] += S[None, :] * G[g][:, J]
        return out.reshape(-1)

    def dipole(self, d: np.ndarray, x: np.ndarray) -> np.ndarray:
        """mu x with mu = -sum_pq d_pq E_pq (spin-summed), mu_c = 0."""
        C = np.asarray(x, np.float64).reshape(self.nsa, self.nsb)
        D = self.apply_E(C)
        return -np.tensordot(np.asarray(d, np.float64).reshape(-1), D, axes=(0, 0)).reshape(-1)
