"""GB300-native nonlocal operator library (after Tian & Engquist, arXiv 1905.08375).

The compute path lives in ``csrc/`` (CUDA for sm_103a, behind the C-ABI declared
in ``include/nl.h``); ``binding`` is a thin ctypes layer over that library with
the same entry-point names.  Importing this package does not load the CUDA
library; ``binding.lib()`` does, and fails loudly when it has not been built.
"""
__all__ = ["binding", "synth"]
