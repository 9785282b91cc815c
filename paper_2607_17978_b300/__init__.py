"""B300-native periodic charge-equilibration (QEq) solver.

The compute path lives in the CUDA library ``libqeq.so`` (``csrc/``) behind a
C ABI (``include/qeq.h``); ``qeq`` is its thin ctypes binding.  ``synth`` draws
seeded synthetic inputs.  Importing the package does not load the library.
"""
