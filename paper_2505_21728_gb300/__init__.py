"""GB300-native Hypercube-Givens Transform (HyGT) library.

The compute path lives in ``csrc/`` (CUDA kernels for sm_103a behind a C-ABI
shared library, ``libhygt.so``); ``hygt`` is the thin Python binding and
``inputs`` the seeded synthetic input generators; ``params`` saves and
loads transform parameters.  Importing the package does
not load the CUDA library; importing ``hygt`` does, and fails loudly if it has
not been built.
"""
__all__ = ["hygt", "inputs", "build", "params"]
