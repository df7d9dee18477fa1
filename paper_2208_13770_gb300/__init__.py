"""GB300-native local Verlet buffer broad phase for soft-sphere DEM.

* ``lvb``     -- ctypes binding of the C-ABI library ``liblvb.so`` (argument
  marshalling only; every step of the path runs in its CUDA kernels).
* ``scenes``  -- seeded synthetic scenes (inputs only).
* ``build``   -- compiles the library for sm_103a with nvcc.

Importing the package loads nothing; ``from paper_2208_13770_gb300 import
lvb`` loads the library and raises if it has not been built.
"""
