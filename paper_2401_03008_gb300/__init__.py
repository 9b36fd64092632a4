"""GB300-native ECHO special-relativistic MHD right-hand-side update.

The compute path is the C-ABI library ``libecho`` (hand-written CUDA for sm_103a,
declared in ``include/echo.h``); :mod:`.echo` is its thin ctypes binding and
:mod:`.workloads` holds the seeded synthetic inputs.
"""
__all__ = ["echo", "workloads"]
