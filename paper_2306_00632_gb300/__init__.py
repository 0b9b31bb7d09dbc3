"""GB300 (sm_103a) TPCG solver for isogeometric Poisson problems in Tucker format.

The compute path is the CUDA library built from ``csrc/`` (C ABI in ``include/tpcg.h``); ``lib`` loads
it with ctypes and ``api`` wraps the entry points with PyTorch-allocated device buffers.
"""
__all__ = ["build", "lib", "api"]
