"""Host-side checks of the C-ABI library that need no GPU.

The library must build, load, and export every entry point declared in
include/kpm.h; host-side argument validation must reject bad inputs before any
device work; without a device, creating a context must fail loudly (no CPU
fallback).
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_07430_gb300 import build
    build.build()
    import paper_2506_07430_gb300 as pkg
    return pkg.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "kpm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kpm_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_are_exported(lib):
    import paper_2506_07430_gb300._lib as L
    names = _declared()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", L.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (kpm_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # the binding declares exactly the header's functions
    assert sorted(L.SIGNATURES) == names
    for n in names:
        getattr(lib, n)


def _call_create(lib, h1, eri, dip, n, na, nb, prec=0):
    h = ctypes.c_void_p()
    st = lib.kpm_create(h1.ctypes.data, eri.ctypes.data, dip.ctypes.data, n, na, nb, prec, None,
                        ctypes.byref(h))
    return st, h


def test_create_rejects_bad_arguments(lib):
    I = synthetic.integrals(4, 2, 2, seed=1)
    h1, eri, dip = I.h1.copy(), I.eri.copy(), I.dipole.copy()
    st, h = _call_create(lib, h1, eri, dip, 4, 2, 5)
    assert st == 1 and not h.value
    assert b"electron" in lib.kpm_last_error(None)
    st, _ = _call_create(lib, h1, eri, dip, 19, 2, 2)
    assert st == 1
    bad = h1.copy()
    bad[0, 1] += 1e-6
    st, _ = _call_create(lib, bad, eri, dip, 4, 2, 2)
    assert st == 1 and b"symmetric" in lib.kpm_last_error(None)
    bad_e = eri.copy()
    bad_e[0, 1, 2, 3] += 1e-6
    st, _ = _call_create(lib, h1, bad_e, dip, 4, 2, 2)
    assert st == 1 and b"symmetry" in lib.kpm_last_error(None)
    st, _ = _call_create(lib, h1, eri, dip, 4, 2, 2, prec=9)
    assert st == 1


def test_null_context_calls_fail_cleanly(lib):
    assert lib.kpm_dim(None) == -1
    assert lib.kpm_nstrings(None, 0) == -1
    assert lib.kpm_sigma(None, None, None, 1) == 1
    assert lib.kpm_recursion_advance(None, 1) == 1
    assert lib.kpm_moments_batch(None, 0, None, 1, None, None, 4, None) == 1
    two_null = (ctypes.c_void_p * 2)(None, None)
    assert lib.kpm_moments_batch(two_null, 2, None, 1, None, None, 4, None) == 1
    assert lib.kpm_recursion_advance_batch(None, 1, 4) == 1
    assert lib.kpm_recursion_advance_batch(two_null, 2, 4) == 1
    a, b = ctypes.c_double(), ctypes.c_double()
    lib.kpm_scale(-3.0, 5.0, 0.01, ctypes.byref(a), ctypes.byref(b))
    assert abs(a.value - 8.0 / 1.99) < 1e-15 and b.value == 1.0


def test_no_device_means_error_not_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    I = synthetic.integrals(4, 2, 2, seed=1)
    st, h = _call_create(lib, I.h1, I.eri, I.dipole, 4, 2, 2)
    assert st == 3 and not h.value
    mu = np.ones(8)
    om = np.zeros(16)
    it = np.zeros(16)
    st = lib.kpm_spectrum(mu.ctypes.data, 8, 1.0, 0.0, 16, 1, om.ctypes.data, it.ctypes.data)
    assert st == 3


def test_binding_refuses_missing_library(tmp_path, monkeypatch):
    import paper_2506_07430_gb300._lib as L
    monkeypatch.setattr(L, "_LIB", None)
    monkeypatch.setattr(L, "_LIBPATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        L.load_library()


def test_batch_bindings_validate_lists_before_any_call():
    import paper_2506_07430_gb300 as pkg
    with pytest.raises(ValueError):
        pkg.moments_batch([], [], 1, [], [], 4)
    with pytest.raises(ValueError):
        pkg.recursion_advance_batch([], 4)

