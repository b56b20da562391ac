"""ctypes declarations of include/kpm.h and a small object wrapper."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "_build", "libkpm.so")
_LIB = None

KPM_OK, KPM_EINVAL, KPM_ENOMEM, KPM_ECUDA, KPM_EBOUNDS, KPM_ETIMEOUT, KPM_ECANCELLED, \
    KPM_EUNSUPPORTED = range(8)
_STATUS = {0: "KPM_OK", 1: "KPM_EINVAL", 2: "KPM_ENOMEM", 3: "KPM_ECUDA", 4: "KPM_EBOUNDS",
           5: "KPM_ETIMEOUT", 6: "KPM_ECANCELLED", 7: "KPM_EUNSUPPORTED"}
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed": 2, "mixed_bf16": 3}

# Every function declared in include/kpm.h with (restype, argtypes).
_P, _I, _I64, _U, _U64, _D = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint,
                              ctypes.c_uint64, ctypes.c_double)
SIGNATURES = {
    "kpm_create": (_I, [_P, _P, _P, _I, _I, _I, _I, _P, _P]),
    "kpm_destroy": (None, [_P]),
    "kpm_last_error": (ctypes.c_char_p, [_P]),
    "kpm_dim": (_I64, [_P]),
    "kpm_nstrings": (_I64, [_P, _I]),
    "kpm_nexc": (_I, [_P, _I]),
    "kpm_string_table": (_I, [_P, _I, _P, _P, _P, _P]),
    "kpm_sigma": (_I, [_P, _P, _P, _I]),
    "kpm_sigma_pauli": (_I, [_P, _P, _P, _I]),
    "kpm_pauli_terms": (_I, [_P, _P, _P]),
    "kpm_apply_dipole": (_I, [_P, _I, _P, _P]),
    "kpm_bounds": (_I, [_P, _I, _U64, _P, _P]),
    "kpm_scale": (None, [_D, _D, _D, _P, _P]),
    "kpm_ground_state": (_I, [_P, _I, _I, _D, _U64, _P, _P, _P]),
    "kpm_moments": (_I, [_P, _P, _U, _D, _D, _I, _P]),
    "kpm_moments_host": (_I, [_P, _P, _U, _D, _D, _I, _P]),
    "kpm_moments_batch": (_I, [_P, _I, _P, _U, _P, _P, _I, _P]),
    "kpm_moments_deflated": (_I, [_P, _P, _D, _U, _D, _D, _I, _P]),
    "kpm_recursion_begin_deflated": (_I, [_P, _P, _D, _U, _D, _D, _I]),
    "kpm_recursion_begin": (_I, [_P, _P, _U, _D, _D, _I]),
    "kpm_recursion_advance": (_I, [_P, _I]),
    "kpm_recursion_advance_batch": (_I, [_P, _I, _I]),
    "kpm_recursion_moments": (_I, [_P, _P, _P]),
    "kpm_spectrum": (_I, [_P, _I, _D, _D, _I, _I, _P, _P]),
    "kpm_spectrum_lorentz": (_I, [_P, _I, _D, _D, _I, _D, _P, _P]),
    "kpm_moments_cross": (_I, [_P, _P, _P, _P, _D, _D, _I, _P]),
    "kpm_synchronize": (_I, [_P]),
    "kpm_profile_enable": (_I, [_P, _I]),
    "kpm_profile_read": (_I, [_P, _P, _P]),
    "kpm_profile_read_rowpass": (_I, [_P, _P, _P]),
    "kpm_graphs_enable": (_I, [_P, _I]),
    "kpm_tuned_params": (_I, [_P, _P, _P]),
    "kpm_tuned_rowpass": (_I, [_P, _P, _P]),
    "kpm_set_rowpass": (_I, [_P, _I, _I]),
    "kpm_rowpass_layout": (_I, [_P, _P, _P]),
    "kpm_set_rowpass_passes": (_I, [_P, _I]),
    "kpm_test_rowpass_stall": (_I, [_P, _I]),
    "kpm_spectrum_static": (_I, [_P, _I, _D, _D, _I, _I, _P, _P, _P]),
    "kpm_server_create": (_I, [_P, _P]),
    "kpm_server_submit": (_I, [_P, _P, _P]),
    "kpm_server_wait": (_I, [_P, _U64, _I, _P]),
    "kpm_server_cancel": (_I, [_P, _U64]),
    "kpm_server_stats": (_I, [_P, _P, _P, _P]),
    "kpm_server_destroy": (None, [_P]),
    "kpm_server_inject_failure": (_I, [_P, _U64, _I]),
    "kpm_launch_count": (_U64, []),
}


class ServerConfig(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("steps_per_round", ctypes.c_int), ("precision", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("h1", _P), ("eri", _P), ("dipole", _P), ("norb", _I), ("nalpha", _I),
                ("nbeta", _I), ("psi0", _P), ("comp_mask", _U), ("a", _D), ("b", _D),
                ("nmoments", _I), ("npoints", _I), ("kernel", _I), ("deflate", _I), ("e0", _D)]


class Result(ctypes.Structure):
    _fields_ = [("moments", _P), ("omega", _P), ("intensity", _P), ("t_queue_s", _D),
                ("t_run_s", _D), ("t_total_s", _D)]


class KPMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return _LIBPATH


def load_library():
    """Load libkpm.so (built by ``paper_2506_07430_gb300.build.build()``); raises if absent."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_LIBPATH):
            raise RuntimeError(f"{_LIBPATH} is missing: run paper_2506_07430_gb300.build.build() "
                               "(the CUDA library is required; there is no fallback)")
        lib = ctypes.CDLL(_LIBPATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def launch_count() -> int:
    return int(load_library().kpm_launch_count())


def _check(st: int, ctx=None):
    if st != KPM_OK:
        msg = load_library().kpm_last_error(ctx).decode()
        raise KPMError(st, msg)


def _np_ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _dev_ptr(t, dtype=None) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch.Tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    return t.data_ptr()


class KPM:
    """One molecule: string tables, integrals and workspaces on the GPU."""

    def __init__(self, h1, eri, dipole, norb: int, nalpha: int, nbeta: int,
                 precision: str = "fp64", stream=None):
        import torch
        lib = load_library()
        self.norb, self.nalpha, self.nbeta = int(norb), int(nalpha), int(nbeta)
        self.precision = precision
        n = self.norb
        h1 = np.ascontiguousarray(h1, dtype=np.float64).reshape(n, n)
        eri = np.ascontiguousarray(eri, dtype=np.float64).reshape(n, n, n, n)
        dipole = np.ascontiguousarray(dipole, dtype=np.float64).reshape(3, n, n)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = lib.kpm_create(_np_ptr(h1), _np_ptr(eri), _np_ptr(dipole), n, self.nalpha,
                            self.nbeta, PRECISIONS[precision], ctypes.c_void_p(stream.cuda_stream),
                            ctypes.byref(h))
        _check(st, None)
        self._h = h
        self.dim = int(lib.kpm_dim(h))
        self.vdtype = torch.float64 if precision == "fp64" else torch.float32

    # -- helpers
    def _lib(self):
        return load_library()

    def close(self):
        if getattr(self, "_h", None):
            self._lib().kpm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nstrings(self, spin: int) -> int:
        return int(self._lib().kpm_nstrings(self._h, spin))

    def nexc(self, spin: int) -> int:
        return int(self._lib().kpm_nexc(self._h, spin))

    def string_table(self, spin: int):
        ns, ne = self.nstrings(spin), self.nexc(spin)
        masks = np.zeros(ns, np.uint32)
        tgt = np.zeros((ns, ne), np.int32)
        pq = np.zeros((ns, ne), np.uint16)
        sgn = np.zeros((ns, ne), np.int8)
        _check(self._lib().kpm_string_table(self._h, spin, _np_ptr(masks), _np_ptr(tgt),
                                            _np_ptr(pq), _np_ptr(sgn)), self._h)
        return masks, tgt, pq, sgn

    def empty(self, ncol: int = 1):
        import torch
        return torch.empty((ncol, self.dim), dtype=self.vdtype, device="cuda")

    def sigma(self, x, y=None):
        """y = H x; x of shape (dim,) or (ncol, dim), dtype float64 (fp64) or float32."""
        ncol = 1 if x.dim() == 1 else x.shape[0]
        if y is None:
            y = x.new_empty(x.shape)
        _check(self._lib().kpm_sigma(self._h, _dev_ptr(x, self.vdtype), _dev_ptr(y, self.vdtype),
                                     ncol), self._h)
        return y

    def sigma_pauli(self, x, y=None):
        """y = H x with H as Jordan-Wigner Pauli strings (kpm_sigma_pauli)."""
        ncol = 1 if x.dim() == 1 else x.shape[0]
        if y is None:
            y = x.new_empty(x.shape)
        _check(self._lib().kpm_sigma_pauli(self._h, _dev_ptr(x, self.vdtype),
                                           _dev_ptr(y, self.vdtype), ncol), self._h)
        return y

    def pauli_terms(self):
        """(number of Pauli strings, number of distinct flip masks)."""
        nt, ng = ctypes.c_int64(), ctypes.c_int()
        _check(self._lib().kpm_pauli_terms(self._h, ctypes.byref(nt), ctypes.byref(ng)), self._h)
        return nt.value, ng.value

    def apply_dipole(self, comp: int, psi, y=None):
        import torch
        if y is None:
            y = torch.empty(self.dim, dtype=self.vdtype, device="cuda")
        _check(self._lib().kpm_apply_dipole(self._h, comp, _dev_ptr(psi, torch.float64),
                                            _dev_ptr(y, self.vdtype)), self._h)
        return y

    def bounds(self, iters: int = 100, seed: int = 2506000):
        lo, hi = ctypes.c_double(), ctypes.c_double()
        _check(self._lib().kpm_bounds(self._h, iters, seed, ctypes.byref(lo), ctypes.byref(hi)),
               self._h)
        return lo.value, hi.value

    def ground_state(self, iters: int = 60, max_cycles: int = 20, tol: float = 1e-9,
                     seed: int = 2506002, out=None):
        """(E0, residual, psi) with psi a CUDA float64 tensor (kpm_ground_state)."""
        import torch
        if out is None:
            out = torch.empty(self.dim, dtype=torch.float64, device="cuda")
        e0, res = ctypes.c_double(), ctypes.c_double()
        _check(self._lib().kpm_ground_state(self._h, iters, max_cycles, tol, seed,
                                            _dev_ptr(out, torch.float64), ctypes.byref(e0),
                                            ctypes.byref(res)), self._h)
        return e0.value, res.value, out

    @staticmethod
    def scale(emin: float, emax: float, eps: float = 0.01):
        a, b = ctypes.c_double(), ctypes.c_double()
        load_library().kpm_scale(emin, emax, eps, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def moments(self, psi0, comp_mask: int, a: float, b: float, nmoments: int,
                check_bounds: bool = True):
        """Moments [ncomp, nmoments]; psi0 is a CUDA float64 tensor or a host ndarray."""
        import torch
        ncomp = bin(comp_mask).count("1")
        out = np.zeros((ncomp, nmoments), np.float64)
        if isinstance(psi0, np.ndarray):
            p = np.ascontiguousarray(psi0, dtype=np.float64)
            st = self._lib().kpm_moments_host(self._h, _np_ptr(p), comp_mask, a, b, nmoments,
                                              _np_ptr(out))
        else:
            st = self._lib().kpm_moments(self._h, _dev_ptr(psi0, torch.float64), comp_mask, a, b,
                                         nmoments, _np_ptr(out))
        if st == KPM_EBOUNDS and not check_bounds:
            return out
        _check(st, self._h)
        return out

    def moments_deflated(self, psi0, e0: float, comp_mask: int, a: float, b: float,
                         nmoments: int, check_bounds: bool = True):
        """Moments [ncomp, nmoments] for an eigenvector psi0 (CUDA float64) of energy e0,
        with the ground-state term in closed form (kpm_moments_deflated)."""
        import torch
        ncomp = bin(comp_mask).count("1")
        out = np.zeros((ncomp, nmoments), np.float64)
        st = self._lib().kpm_moments_deflated(self._h, _dev_ptr(psi0, torch.float64), e0,
                                              comp_mask, a, b, nmoments, _np_ptr(out))
        if st == KPM_EBOUNDS and not check_bounds:
            return out
        _check(st, self._h)
        return out

    def moments_cross(self, psi0, op_a, op_b, a: float, b: float, nmoments: int,
                      check_bounds: bool = True):
        """Omega_n = <0|A T_n(H~) B|0> for one-body A = sum op_a E, B = sum op_b E
        (symmetric n x n host matrices) (kpm_moments_cross)."""
        import torch
        n = self.norb
        oa = np.ascontiguousarray(op_a, dtype=np.float64).reshape(n, n)
        ob = np.ascontiguousarray(op_b, dtype=np.float64).reshape(n, n)
        out = np.zeros(nmoments, np.float64)
        st = self._lib().kpm_moments_cross(self._h, _dev_ptr(psi0, torch.float64), _np_ptr(oa),
                                           _np_ptr(ob), a, b, nmoments, _np_ptr(out))
        if st == KPM_EBOUNDS and not check_bounds:
            return out
        _check(st, self._h)
        return out

    def recursion_begin(self, psi0, comp_mask: int, a: float, b: float, max_moments: int,
                        e0: float | None = None):
        """Start a resumable recursion; with e0, the deflated form (psi0 an eigenvector)."""
        import torch
        self._rec_ncomp = bin(comp_mask).count("1")
        self._rec_max = max_moments
        if e0 is None:
            st = self._lib().kpm_recursion_begin(self._h, _dev_ptr(psi0, torch.float64),
                                                 comp_mask, a, b, max_moments)
        else:
            st = self._lib().kpm_recursion_begin_deflated(self._h, _dev_ptr(psi0, torch.float64),
                                                          e0, comp_mask, a, b, max_moments)
        _check(st, self._h)

    def recursion_advance(self, nsteps: int):
        _check(self._lib().kpm_recursion_advance(self._h, nsteps), self._h)

    def synchronize(self):
        _check(self._lib().kpm_synchronize(self._h), self._h)

    def tuned_params(self):
        """Autotuner choices: (rasterisation group of the beta GEMM, of the alpha GEMM)."""
        gb, ga = ctypes.c_int(), ctypes.c_int()
        _check(self._lib().kpm_tuned_params(self._h, ctypes.byref(gb), ctypes.byref(ga)), self._h)
        return gb.value, ga.value

    def tuned_rowpass(self):
        """Autotuner choices of the row pass: (A stages, L2 prefetch distance in tiles)."""
        st, pf = ctypes.c_int(), ctypes.c_int()
        _check(self._lib().kpm_tuned_rowpass(self._h, ctypes.byref(st), ctypes.byref(pf)), self._h)
        return st.value, pf.value

    def set_rowpass(self, stages: int, prefetch: int):
        """Pins the row pass's A stages and prefetch distance (kpm_set_rowpass)."""
        _check(self._lib().kpm_set_rowpass(self._h, int(stages), int(prefetch)), self._h)

    def rowpass_layout(self):
        """(wide, passes) of the row pass (kpm_rowpass_layout)."""
        w, np_ = ctypes.c_int(), ctypes.c_int()
        _check(self._lib().kpm_rowpass_layout(self._h, ctypes.byref(w), ctypes.byref(np_)), self._h)
        return bool(w.value), np_.value

    def set_rowpass_passes(self, passes: int):
        """Wide row-pass layout with this many passes (0: automatic)."""
        _check(self._lib().kpm_set_rowpass_passes(self._h, int(passes)), self._h)

    def test_rowpass_stall(self, on: bool = True):
        """Testing aid: the next tensor-core row pass stalls until its bounded waits
        run out (kpm_test_rowpass_stall)."""
        _check(self._lib().kpm_test_rowpass_stall(self._h, 1 if on else 0), self._h)

    def graphs_enable(self, on: bool = True):
        _check(self._lib().kpm_graphs_enable(self._h, 1 if on else 0), self._h)

    def profile_enable(self, on: bool = True):
        _check(self._lib().kpm_profile_enable(self._h, 1 if on else 0), self._h)

    def profile_read(self):
        """(summed ms, count) of H applications since the last read."""
        ms, cnt = ctypes.c_double(), ctypes.c_int()
        _check(self._lib().kpm_profile_read(self._h, ctypes.byref(ms), ctypes.byref(cnt)), self._h)
        return ms.value, cnt.value

    def profile_read_rowpass(self):
        """(summed ms, count) of tensor-core row-pass launches since the last read."""
        ms, cnt = ctypes.c_double(), ctypes.c_int()
        _check(self._lib().kpm_profile_read_rowpass(self._h, ctypes.byref(ms), ctypes.byref(cnt)),
               self._h)
        return ms.value, cnt.value

    def recursion_moments(self):
        out = np.zeros((self._rec_ncomp, self._rec_max), np.float64)
        nm = ctypes.c_int()
        st = self._lib().kpm_recursion_moments(self._h, _np_ptr(out), ctypes.byref(nm))
        if st not in (KPM_OK, KPM_EBOUNDS):
            _check(st, self._h)
        k = nm.value
        return out.reshape(-1)[: self._rec_ncomp * k].reshape(self._rec_ncomp, k)


class Server:
    """Continuous-batching spectrum server (kpm_server_*)."""

    def __init__(self, mem_budget_bytes: int, max_slots: int = 8, steps_per_round: int = 16,
                 precision: str = "mixed"):
        lib = load_library()
        cfg = ServerConfig(int(mem_budget_bytes), int(max_slots), int(steps_per_round),
                           PRECISIONS[precision])
        h = ctypes.c_void_p()
        _check(lib.kpm_server_create(ctypes.byref(cfg), ctypes.byref(h)), None)
        self._h = h
        self._pending = {}

    def submit(self, h1, eri, dipole, norb, nalpha, nbeta, psi0, comp_mask, a, b, nmoments,
               npoints=2048, kernel="jackson", e0=None):
        """Queue a request; with e0 (psi0 an eigenvector of that energy) the recursion
        runs deflated (kpm_moments_deflated)."""
        keep = [np.ascontiguousarray(h1, dtype=np.float64),
                np.ascontiguousarray(eri, dtype=np.float64),
                np.ascontiguousarray(dipole, dtype=np.float64),
                np.ascontiguousarray(psi0, dtype=np.float64)]
        r = Request(_np_ptr(keep[0]), _np_ptr(keep[1]), _np_ptr(keep[2]), norb, nalpha, nbeta,
                    _np_ptr(keep[3]), comp_mask, a, b, nmoments, npoints,
                    KERNELS[kernel], 0 if e0 is None else 1,
                    0.0 if e0 is None else float(e0))
        rid = ctypes.c_uint64()
        _check(load_library().kpm_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)), None)
        self._pending[rid.value] = (bin(comp_mask).count("1"), nmoments, npoints)
        return rid.value

    def wait(self, rid: int, timeout_ms: int = 600000, allow_ebounds: bool = False):
        ncomp, nm, npts = self._pending[rid]
        mom = np.zeros((ncomp, nm))
        om = np.zeros(npts)
        it = np.zeros(npts)
        res = Result(_np_ptr(mom), _np_ptr(om), _np_ptr(it), 0.0, 0.0, 0.0)
        st = load_library().kpm_server_wait(self._h, rid, timeout_ms, ctypes.byref(res))
        if st == KPM_ETIMEOUT:
            _check(st, None)
        del self._pending[rid]
        if not (st == KPM_OK or (allow_ebounds and st == KPM_EBOUNDS)):
            _check(st, None)
        return {"moments": mom, "omega": om, "intensity": it, "t_queue_s": res.t_queue_s,
                "t_run_s": res.t_run_s, "t_total_s": res.t_total_s, "status": st}

    def inject_failure(self, rid: int, status: int):
        """Testing aid: the next advance of request rid fails with `status`."""
        _check(load_library().kpm_server_inject_failure(self._h, rid, status), None)

    def cancel(self, rid: int):
        _check(load_library().kpm_server_cancel(self._h, rid), None)

    def stats(self):
        mem, res, q = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
        _check(load_library().kpm_server_stats(self._h, ctypes.byref(mem), ctypes.byref(res),
                                               ctypes.byref(q)), None)
        return {"mem_used": mem.value, "resident": res.value, "queued": q.value}

    def close(self):
        if getattr(self, "_h", None):
            load_library().kpm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def moments_batch(kpms, psi0s, comp_mask: int, a, b, nmoments: int, check_bounds: bool = True):
    """Moments of several molecules in batched launches (kpm_moments_batch).

    kpms: FP64 or FP32 KPM contexts (one precision); psi0s: CUDA float64 tensors;
    a, b: per-molecule rescaling.  Returns [len(kpms), ncomp, nmoments]."""
    import torch
    count = len(kpms)
    if count == 0 or len(psi0s) != count or len(a) != count or len(b) != count:
        raise ValueError("kpms, psi0s, a and b need the same non-zero length")
    ncomp = bin(comp_mask).count("1")
    out = np.zeros((count, ncomp, nmoments), np.float64)
    ctxs = (ctypes.c_void_p * count)(*[k._h for k in kpms])
    psis = (ctypes.c_void_p * count)(*[_dev_ptr(p, torch.float64) for p in psi0s])
    av = np.ascontiguousarray(a, dtype=np.float64)
    bv = np.ascontiguousarray(b, dtype=np.float64)
    st = load_library().kpm_moments_batch(ctxs, count, psis, comp_mask, _np_ptr(av), _np_ptr(bv),
                                          nmoments, _np_ptr(out))
    if st == KPM_EBOUNDS and not check_bounds:
        return out
    _check(st, kpms[0]._h)
    return out


def recursion_advance_batch(kpms, nsteps: int):
    """kpm_recursion_advance_batch: advance every context's resumable recursion
    by nsteps in batched launches (asynchronous)."""
    count = len(kpms)
    if count == 0:
        raise ValueError("empty context list")
    ctxs = (ctypes.c_void_p * count)(*[k._h for k in kpms])
    _check(load_library().kpm_recursion_advance_batch(ctxs, count, nsteps), kpms[0]._h)


KERNELS = {"none": 0, "jackson": 1, "lorentz": 2}


def spectrum(moments, a: float, b: float, npoints: int = 2048, kernel: str = "jackson",
             lam: float | None = None):
    """(omega ascending, intensity per unit energy) on the Chebyshev nodes; kernel
    "jackson", "lorentz" (parameter lam, default KPM_LORENTZ_LAMBDA) or "none"."""
    lib = load_library()
    mu = np.ascontiguousarray(moments, dtype=np.float64).reshape(-1)
    om = np.zeros(npoints, np.float64)
    it = np.zeros(npoints, np.float64)
    if kernel == "lorentz" and lam is not None:
        st = lib.kpm_spectrum_lorentz(_np_ptr(mu), len(mu), a, b, npoints, float(lam),
                                      _np_ptr(om), _np_ptr(it))
    else:
        st = lib.kpm_spectrum(_np_ptr(mu), len(mu), a, b, npoints, KERNELS[kernel],
                              _np_ptr(om), _np_ptr(it))
    _check(st, None)
    return om, it
