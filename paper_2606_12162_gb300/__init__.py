"""GB300-native explicit finite-volume step for the hyperbolic Serre-Green-Naghdi
systems (mbHSGN, HSGN) with the transition to the shallow water equations.

The compute path is the CUDA library built from csrc/ (sm_103a) behind the C ABI
of include/sgn.h; `paper_2606_12162_gb300.sgn` is its ctypes binding.  Importing
this package does not load the library; `sgn.load()` does, and raises if the
library has not been built.
"""
__all__ = ["sgn", "workloads"]
