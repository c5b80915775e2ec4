"""GB300-native shape-constrained gravitational point-cloud registration.

The compute path is the CUDA library libscgr.so (C ABI in include/scgr.h),
reached from Python through ``paper_1902_01061_gb300.scgr``.  ``synth`` holds
the seeded synthetic input generators; ``build`` compiles the library.
"""
