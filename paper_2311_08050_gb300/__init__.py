"""GB300-native (sm_103a) dense INLA theta-evaluation engine.

The compute path is the C-ABI library ``libinla.so`` (CUDA kernels in ``csrc/``);
``inla.py`` is its thin ctypes binding.  ``synth.py`` holds the seeded synthetic
workloads.  Importing the package loads nothing: the library is loaded on first use.
"""
__all__ = ["synth", "inla"]
