"""GB300-native muon-tomography posterior evaluation and batched MCMC.

``paper_2603_28907_gb300.mt`` is the ctypes binding of ``libmt.so`` (the C-ABI
declared in ``include/mt.h``); ``paper_2603_28907_gb300.workloads`` builds the
seeded synthetic problems.  Importing the package loads neither.
"""
__all__ = ["mt", "workloads"]
