"""GB300-native (sm_103a) Wilson-fermion multi-mass solver library.

The compute path is the C-ABI shared library ``libwilson.so`` built from
``csrc/`` (see ``include/wilson.h``); ``api`` is a thin ctypes binding that
marshals torch device tensors into it.  ``synth`` generates the seeded
synthetic gauge fields and sources.
"""
__all__ = ["synth"]
