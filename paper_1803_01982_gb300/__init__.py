"""GB300-native Flip-Flop SRQR (Feng, Xiao & Gu, arXiv 1803.01982): a rank-k
approximate SVD behind a small C ABI (``include/ffsrqr.h``).

Submodules:
  ``ffsrqr``  -- ctypes binding of ``_lib/libffsrqr.so`` (import fails if it is not built)
  ``build``   -- nvcc build of ``csrc/`` for sm_103a
  ``synth``   -- seeded synthetic test matrices (no factorisation arithmetic)
"""
