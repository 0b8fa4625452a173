"""GB300-native immersed-boundary acoustic finite differences (Caunt et al.).

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through ``paper_2309_03600_gb300.ib`` (a ctypes binding with the same
entry-point names as ``include/ib.h``).  ``inputs`` builds seeded synthetic
workloads.  Importing this package does not load the library; the first call
into ``ib`` does, and fails loudly if it has not been built.
"""
__all__ = ["ib", "inputs"]
