"""GB300-native hot path of known-pose, diagonally preconditioned SGD for
cryo-EM refinement (Toader, Brubaker & Lederman, arXiv 2311.16100).

Submodules (imported lazily; nothing here loads the CUDA library):
  native  -- ctypes declarations of libcryosgd (include/cryosgd.h)
  ops     -- thin torch binding: Handle, Geometry, CTF, SGDState
  synth   -- seeded synthetic inputs (volumes, rotations, defocus)
  build   -- nvcc build of libcryosgd.so for sm_103a
"""
