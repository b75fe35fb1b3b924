"""GB300-native real-time CCSD (RT-CCSD) propagation library.

The compute path lives in the CUDA shared library ``librtcc.so`` built from
``csrc/`` and is reached through the C-ABI declared in ``include/rtcc.h``;
``rtcc.py`` is a thin ctypes binding with the same names.  Importing this
package does not load the library; ``paper_2205_05175_gb300.rtcc`` does, and it
raises if the library is missing (there is no CPU fallback).
"""
__all__ = ["synth"]
