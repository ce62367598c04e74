"""GB300-native split-step Crank-Nicolson step of the 3D dipolar Gross-Pitaevskii equation.

The compute path is the CUDA library ``csrc/`` builds (``libdgpe.so``, C-ABI declared in
``include/dgpe.h``); ``abi`` is its thin ctypes binding.  Importing this package does not
load the library; ``abi.load()`` does, and raises if it is missing.
"""
__all__ = ["abi", "inputs"]
