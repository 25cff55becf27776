"""FP64 CPU oracle of the particle -> IFU cube forward model (arXiv 2412.08265).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the library. It shares no code with the
CUDA path. ``oracle.core`` wraps the plain C implementation
(``rubix_oracle.c``); the test suite's ``tests/_brute.py`` is an independent
NumPy/SciPy restatement for tiny inputs that pins the C oracle.
"""
from .core import (build, forward, forward_parts, orient, spaxel_keys, stable_sort, deposit,
                   psf, lsf, psf_lsf_at, gradient, gauss_kernel, kernel_radius, C_KMS)

__all__ = ["build", "forward", "forward_parts", "orient", "spaxel_keys", "stable_sort",
           "deposit", "psf", "lsf", "psf_lsf_at", "gradient", "gauss_kernel",
           "kernel_radius", "C_KMS"]
