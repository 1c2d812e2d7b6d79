"""GB300-native stage-system solver for fully implicit Runge-Kutta time steps
of discontinuous Galerkin discretisations (Pazner & Persson, arXiv 1701.07181).

The compute path is ``libirk_gb300.so`` (hand-written CUDA for sm_103a behind
a C ABI, declared in ``include/irk_gb300.h``); ``paper_1701_07181_gb300.irk``
is its thin ctypes binding.  ``inputs`` generates seeded synthetic workloads.
Importing this package loads nothing; the library is loaded on first use.
"""
__all__ = ["inputs", "irk"]
