"""GB300-native low-rank evaluation of the multi-particle Smoluchowski system.

The compute path is the C-ABI library ``libsag.so`` (hand-written sm_103a CUDA,
declared in ``include/sag.h``); ``paper_1905_09071_gb300.sag`` is its thin
ctypes binding. Importing this package loads nothing: the library is opened on
first use and raises if it is missing.
"""
__all__ = ["sag", "workloads"]
