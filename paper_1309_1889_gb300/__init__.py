"""GB300-native multilevel summation method (MSM) with velocity Verlet and parareal.

The compute path lives in ``libmsm_gb300.so`` (hand-written sm_103a CUDA kernels
behind a C ABI, declared in ``include/msm.h``).  This package holds the thin
ctypes binding (``api``), the build step (``build``) and the seeded synthetic
input generator (``inputs``).  Importing the package does not load the library;
the first call into ``api`` does, and raises if it is missing.
"""

__all__ = ["api", "inputs", "build"]
