"""GB300-native polynomial preconditioned Arnoldi (Embree, Loe & Morgan).

The compute path lives in the CUDA/C++ shared library under ``csrc/`` behind
the C-ABI declared in ``include/pp.h``; :mod:`.pp` is its ctypes binding.
Importing this package does not load the library; ``from
paper_1806_08020_gb300 import pp`` does, and fails loudly when it is missing.
"""
