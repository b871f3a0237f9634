"""GB300-native AFN-preconditioned CG for regularized kernel systems.

The compute path is the C-ABI library ``libafn.so`` (hand-written sm_103a CUDA
kernels behind ``include/afn.h``); :mod:`paper_2304_05460_gb300.afn` is its
thin Python binding and :mod:`paper_2304_05460_gb300.inputs` draws the seeded
synthetic workloads.
"""
__all__ = ["afn", "inputs"]
