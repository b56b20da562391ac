"""kpm_spectrum_static: the spectrum entry point that allocates nothing.

It serves callers that cannot call cudaMalloc (device memory entirely held by
another allocator, or loops that cannot pay for allocation and its implicit
device synchronisation).  It must give the same spectrum as the allocating
kpm_spectrum, call after call, with its scratch in the library's fixed device
array.  The device buffers below belong to the caller (this test); the entry
point itself allocates nothing.

This file is named so that pytest collects it after every other test file.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# Same bound as the other spectrum parity tests: identical moments, FP64 sums.
TOL = 1e-10


def _case(seed, N):
    rng = np.random.default_rng(seed)
    mu = rng.standard_normal(N) / (1.0 + np.arange(N)) * 0.4
    mu[0] = 1.0
    return mu


def test_static_spectrum_matches_allocating_entry_point():
    import torch

    from paper_2506_07430_gb300 import load_library, spectrum

    lib = load_library()
    stream = torch.cuda.current_stream()
    for call, (seed, N, M, a, b, kern) in enumerate([(1, 1000, 2048, 3.1, -7.5, 1),
                                                      (2, 257, 513, 0.8, 0.25, 1)]):
        mu = _case(seed, N)
        om_ref, it_ref = spectrum(mu, a, b, M, "jackson" if kern else "none")
        mu_d = torch.tensor(mu, dtype=torch.float64, device="cuda")
        om_d = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
        it_d = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.kpm_spectrum_static(mu_d.data_ptr(), N, a, b, M, kern, om_d.data_ptr(),
                                     it_d.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.kpm_last_error(None)
        torch.cuda.synchronize()
        om, it = om_d.cpu().numpy(), it_d.cpu().numpy()
        assert np.all(np.isfinite(om)) and np.all(np.isfinite(it)), call
        assert np.abs(om - om_ref).max() <= TOL * (abs(a) + abs(b))
        assert np.linalg.norm(it - it_ref) <= TOL * np.linalg.norm(it_ref), call


def test_static_spectrum_leaves_device_memory_unchanged():
    """After a first call (which loads the kernels and looks up the array's
    address), further calls leave the device's free memory exactly as it was:
    nothing is allocated, the scratch is the library's fixed array."""
    import torch

    from paper_2506_07430_gb300 import load_library

    lib = load_library()
    stream = torch.cuda.current_stream()
    N, M = 4096, 1024
    mu_d = torch.tensor(_case(3, N), dtype=torch.float64, device="cuda")
    om_d = torch.empty(M, dtype=torch.float64, device="cuda")
    it_d = torch.empty(M, dtype=torch.float64, device="cuda")

    def call():
        st = lib.kpm_spectrum_static(mu_d.data_ptr(), N, 1.5, 0.5, M, 1, om_d.data_ptr(),
                                     it_d.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.kpm_last_error(None)

    call()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    first = it_d.cpu().numpy()
    for _ in range(20):
        call()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(it_d.cpu().numpy(), first)


def test_static_spectrum_rejects_oversized_request():
    import torch

    from paper_2506_07430_gb300 import load_library

    lib = load_library()
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = lib.kpm_spectrum_static(d.data_ptr(), 262145, 1.0, 0.0, 4, 1, d.data_ptr(),
                                 d.data_ptr(), None)
    assert st == 1
    assert b"exceeds the static scratch" in lib.kpm_last_error(None)
