"""GB300 (sm_103a) SH-FFT estimator of power-spectrum multipoles with a moving line of sight.

The compute lives in libpspec.so (CUDA kernels behind the C ABI of include/pspec.h); this
package holds its build script and a thin ctypes binding.
"""
from .pspec import Estimator, PspecError, wedges, load  # noqa: F401

__all__ = ["Estimator", "PspecError", "wedges", "load"]
