"""B300-native (sm_103a) CBAA super-host detector.

Submodules:
  traffic  -- seeded synthetic edge-router traffic (numpy only)
  cbaa     -- ctypes binding of libcbaa.so (loads the CUDA library; no fallback)
  build    -- nvcc build of libcbaa.so
"""
__all__ = ["traffic", "cbaa", "build"]
