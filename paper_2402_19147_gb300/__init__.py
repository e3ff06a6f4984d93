"""GB300 (sm_103a) QMCUR hot path: quaternion CUR low-rank approximation.

The compute runs in ``libqmcur.so`` (CUDA, C ABI, declared in include/qmcur.h);
``paper_2402_19147_gb300.qmcur`` is a thin ctypes binding with the same names.
Importing this package does not load the library; ``qmcur.lib()`` does, and it
raises if the library has not been built (there is no CPU fallback).
"""
