"""GB300-native (sm_103a) Faster-GS training step.

The compute path is the C-ABI library ``libfastergs.so`` built from
``csrc/`` (see ``include/fastergs.h``); :mod:`.binding` is its thin ctypes
binding and :mod:`.train` the PyTorch-facing step built on it.  Importing
this package does not load the library; the first call into the binding
does, and fails loudly when the library is missing.
"""
__all__ = ["binding", "scenes", "train"]
