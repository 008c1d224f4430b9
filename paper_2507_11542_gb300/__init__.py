"""GB300-native (sm_103a) Hamilton-Jacobi level-set step after LevelSetPy (arXiv 2507.11542).

The compute path is libhj.so (CUDA kernels behind the C ABI of include/hj.h);
``_lib`` is its thin ctypes binding, ``solver`` a torch-tensor convenience
layer over it, ``workloads`` the seeded synthetic inputs.
"""
__all__ = ["build", "workloads"]
