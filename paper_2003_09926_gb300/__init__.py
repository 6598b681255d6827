"""GB300-native (sm_103a) implementation of the per-stage residual and explicit
5-stage Runge-Kutta update of the filtered compressible Navier-Stokes (LES)
equations on a structured curvilinear grid (arXiv 2003.09926, Sections 3-4).

The compute path is the CUDA library ``libjz.so`` behind the C ABI in
``include/jz.h``; ``jz`` is its thin Python binding, ``workloads`` holds the
synthetic grid/flow configurations and ``serve`` the request loop.
"""
__all__ = ["jz", "workloads", "build"]
