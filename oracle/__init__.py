"""FP64 CPU oracle for the spherical-harmonic FFT multipole estimator.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package. The product path (the CUDA library and its
Python binding) never imports, calls or links anything here, and this package imports
nothing from the product.

Modules
-------
``estimator``  the estimator itself (Sec. 2.1 eqs. FKP-density, Pell-ours, Fell, real-Ylm;
               Sec. 2.3 painting, interlacing, compensation; Sec. 2.2 wedges eqs. wedge-est,
               Lbar), written as plainly as possible in NumPy/SciPy FP64.
``brute``      independent routes used to pin the estimator: the direct particle sum of the
               local plane-parallel estimator (eq. Pell-yama), the Cartesian decomposition
               for l <= 4 (Sec. 2.1), an O(N^6) DFT, a per-particle loop paint, and the
               alias sums of the mass-assignment windows.

Parity status: every function is pinned by a ``-m "not gpu"`` test against something
other than itself (see tests/test_oracle_*.py); none is "parity unpinned".
"""
