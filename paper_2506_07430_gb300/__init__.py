"""GB300-native kernel polynomial method for dipole absorption spectra.

Thin ctypes binding over the C-ABI library ``libkpm.so`` (``include/kpm.h``).
Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    KPM,
    KPMError,
    PRECISIONS,
    Server,
    launch_count,
    library_path,
    load_library,
    moments_batch,
    recursion_advance_batch,
    spectrum,
)

__all__ = ["KPM", "KPMError", "PRECISIONS", "Server", "moments_batch", "recursion_advance_batch",
           "spectrum", "launch_count", "load_library", "library_path"]
