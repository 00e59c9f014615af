"""GB300-native hot path of time-dependent Hubbard exact diagonalisation.

The compute path lives in ``csrc/`` (CUDA kernels for sm_103a + host C++ +
the C ABI declared in ``include/ed.h``), built in-tree into
``_lib/libhubbard_ed.so`` by ``build.py``; ``ed`` is its ctypes binding.
"""
__all__ = ["ed", "build"]
