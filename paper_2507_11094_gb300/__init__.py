"""GB300-native dynamic single-source shortest paths.

The compute path is ``libsp.so`` (hand-written sm_103a CUDA kernels behind a
C ABI, ``include/sp.h``); :mod:`paper_2507_11094_gb300.sp` is its thin ctypes
binding.  :mod:`paper_2507_11094_gb300.workloads` holds the seeded synthetic
inputs.  Importing the package does not load CUDA; the binding loads the
library on first use and raises if it is missing.
"""

__all__ = ["sp", "workloads"]
