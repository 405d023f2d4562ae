"""GB300-native Mojette erasure code (forward / inverse Mojette transform over GF(2)).

The compute path is the CUDA library ``libmojette.so`` (sources in ``csrc/``,
C ABI in ``include/mojette.h``); ``binding`` wraps it with ctypes. Importing
this package does not load the library: ``binding`` does, on first use, and
raises if it cannot.
"""
__all__ = ["binding", "inputs"]
