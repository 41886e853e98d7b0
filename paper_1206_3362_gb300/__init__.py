"""GB300-native FWBF (fast weighted bit-flipping) LDPC decoding.

The decoder runs in hand-written sm_103a CUDA kernels behind the C ABI of
``libfwbf.so`` (declared in ``include/fwbf.h``); :mod:`.fwbf` is a thin ctypes
binding with the same entry-point names.  :mod:`.inputs` builds seeded codes and
channel values.
"""
__all__ = ["fwbf", "inputs"]
