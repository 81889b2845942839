"""Batched spherical harmonic transforms on HEALPix grids for B300 (sm_103a).

The compute path lives in ``libsht.so`` (hand-written CUDA behind a C ABI,
see ``include/sht.h``); ``paper_2208_10154_b300.sht`` is the thin ctypes
binding. Importing this package does not load the library; the first call
into ``sht`` does, and fails loudly if it is missing.
"""
__all__ = ["inputs"]
