"""GB300-native FAS multigrid with local spectral coarsening for heterogeneous nonlinear diffusion.

`build` compiles the CUDA/C++ library in-tree; `nlmg` is the ctypes binding of its C ABI (include/nlmg.h).
"""
