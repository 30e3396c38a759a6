"""Plain FP64 CPU oracle of the DGSEM hot path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never uses it.
"""
from .oracle import (Oracle, build, lib_path, basis, gauss_basis, ec_flux, llf_flux, roe_flux, log_mean,  # noqa: F401
                     rk_coeffs, rk14_coeffs, count_ec_flux_ops, set_threads, persson_field)
