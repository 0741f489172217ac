"""GB300-native ghost-cell sharp-interface immersed-boundary fractional-step
solver (arxiv 2505.17287, Sections 2.1-2.2): CUDA kernels for sm_103a behind
the C ABI of include/ibm.h, with a thin ctypes binding (``ibm``), seeded
input generators (``synth``) and the build script (``build``).

Importing the package loads nothing compiled; ``paper_2505_17287_gb300.ibm``
loads libibm.so and raises when it is missing.
"""
__all__ = ["ibm", "synth", "build"]
