"""GB300-native levelwise wavelet tree construction (levelWT).

The library is the CUDA shared object built from ``csrc/``; ``wt`` is its
Python binding (argument marshalling only).  Importing this package loads
nothing; the first call into ``wt`` loads the library and fails loudly when it
is missing.
"""
