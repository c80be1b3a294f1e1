"""Reverse-mode gradients of data-parallel functions on GB300 (sm_103a).

The compute path lives in the C-ABI library ``libkg.so`` (CUDA kernels under
``csrc/``); :mod:`._lib` is its thin ctypes binding.  Importing this package
loads nothing; the library is opened on first use and a missing library is an
error, never a fallback.
"""
__all__ = ["workloads"]
