"""GB300-native ensemble engine for the reduced-precision Gillespie direct method.

The simulation runs in hand-written CUDA kernels for sm_103a behind a C ABI
(``include/ssa.h``); ``paper_2605_00479_gb300.ssa`` is the thin ctypes binding.
Importing the package does not load the CUDA library; ``ssa.lib()`` does, and
raises if it has not been built.
"""
