"""GB300-native MG-GLAM scalar-field multigrid (arXiv:2110.00328).

The compute path is the C-ABI library ``libmgglam.so`` (hand-written sm_103a
CUDA kernels, declared in ``include/mgglam.h``); ``binding`` marshals torch
device tensors into it.  ``inputs`` holds the seeded synthetic workload
generators.  Importing this package does not load the CUDA library; the
binding loads it on first use and raises if it is missing.
"""
__all__ = ["inputs", "binding"]
