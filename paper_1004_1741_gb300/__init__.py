"""GB300-native 3D 7-point Jacobi and lexicographic Gauss-Seidel smoothers with
temporal blocking (after Treibig, Wellein, Hager, arXiv:1004.1741).

Submodules:
  capi       Python binding of the C ABI (include/stencil.h); needs the CUDA library.
  build      builds _lib/libstencil.so for sm_103a.
  workloads  seeded synthetic grids (no smoother arithmetic).
"""
__all__ = ["capi", "build", "workloads"]
