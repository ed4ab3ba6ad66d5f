"""GB300-native (sm_103a) even-odd preconditioned domain-wall fermion CG solver.

The compute path lives in the CUDA library built from ``csrc/`` (C-ABI declared in
``include/dwf.h``); ``dwf`` is its thin ctypes binding and ``inputs`` the seeded
synthetic input generators.  Nothing is loaded at import time.
"""
