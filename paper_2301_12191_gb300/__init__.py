"""GB300-native multi-resolution inter analysis (integer full-search ME +
8x8 SATD quadtree split decision, independent and dependent ladder rungs).

The compute path is the CUDA library ``libladder.so`` behind the C ABI in
``include/ladder.h``; ``paper_2301_12191_gb300.ladder`` is its thin ctypes
binding.  Importing this package loads nothing; the binding loads the library
on first use and raises if it is missing.
"""
__all__ = ["ladder", "synth"]
