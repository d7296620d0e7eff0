"""GB300-native Gaussian belief propagation (GaBP) solver for symmetric Ax = b.

The compute path is the C-ABI library ``libgabp.so`` (hand-written CUDA for
sm_103a, declared in ``include/gabp.h``); ``paper_0810_1119_gb300.gabp`` is the
thin ctypes binding over it.  ``paper_0810_1119_gb300.workloads`` builds the
seeded synthetic inputs.  Importing the package itself loads nothing.
"""
__all__ = ["gabp", "workloads"]
