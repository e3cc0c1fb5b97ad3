"""GB300-native Triggered Cells Method (Naeh, arXiv:1702.00216).

The compute path is the CUDA library built from ``csrc/`` (C ABI declared in
``include/tcm.h``); ``tcm`` is its thin ctypes binding and ``workloads`` the
seeded synthetic inputs.
"""
__all__ = ["tcm", "workloads"]
