"""GB300-native collision core for collisional-plasma PIC (arXiv 2508.06771).

The compute path is the CUDA shared library ``libltpc.so`` built from ``csrc/``
behind the C ABI declared in ``include/ltpc.h``; ``ltpc.py`` is a thin ctypes
binding with the same names.  ``workloads.py`` draws seeded synthetic inputs.
Importing the package loads nothing; ``ltpc`` loads the library on first use
and raises if it is missing (there is no CPU fallback).
"""
__all__ = ["workloads", "ltpc"]
