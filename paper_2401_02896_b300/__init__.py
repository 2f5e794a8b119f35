"""B300-native per-ray higher-order SPH field reconstruction and DVR (arXiv 2401.02896).

Modules:
  sphdvr     -- ctypes binding of libsphdvr (the C ABI in include/sphdvr.h);
                importing it loads lib/libsphdvr.so and raises if it is missing.
  synthetic  -- seeded synthetic particle sets, cameras and transfer functions.
  _build     -- nvcc build of libsphdvr.so for sm_103a.
"""
