"""GB300-native (sm_103a) conservative spectral Boltzmann collision operator.

The compute path is the C-ABI library ``libcs`` (CUDA, ``csrc/``), declared in
``include/cs.h``; ``api`` is its thin Python binding (argument marshalling
only).  Importing this package loads nothing: ``api`` loads the library on
first use and raises if it is missing.
"""
__all__ = ["api", "inputs", "build"]
