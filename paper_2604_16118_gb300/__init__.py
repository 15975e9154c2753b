"""GB300-native block-sparse MPS eigensolver (C ABI in include/bsmps.h).

``native`` is the ctypes binding of libbsmps.so; ``build`` compiles it for
sm_103a.  Importing the package itself loads nothing.
"""
