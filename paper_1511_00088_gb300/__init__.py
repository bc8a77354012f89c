"""GB300-native even-odd staggered CG (mixed precision) behind a C-ABI library.

Submodules:
  stag   -- ctypes binding of libstag.so (same names as the C ABI in include/stag.h)
  synth  -- seeded synthetic gauge fields and sources
  build  -- nvcc build of the CUDA library for sm_103a
"""
__all__ = ["stag", "synth", "build"]
