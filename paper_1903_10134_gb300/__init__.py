"""GB300-native many-body DPD (mDPD) hot path, after arXiv:1903.10134.

The compute runs in hand-written sm_103a CUDA kernels behind a C ABI
(``include/mdpd.h``); ``paper_1903_10134_gb300.mdpd`` is the thin ctypes
binding and ``paper_1903_10134_gb300.inputs`` the seeded workload generators.
Nothing is loaded at import time.
"""
__all__ = ["inputs", "mdpd"]
