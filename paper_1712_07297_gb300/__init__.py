"""GB300 hierarchical sparse solver (arXiv 1712.07297, LoRaSp-style low-rank
elimination) -- CUDA library ``libhsolve.so`` with a thin ctypes binding.

Submodules
----------
inputs   seeded synthetic problems (no solver arithmetic)
build    nvcc build of the library (sm_103a)
hsolve   ctypes binding of the C-ABI declared in include/hsolve.h
"""
