"""GB300-native TFHE gate bootstrapping (blind rotation, sample extraction,
key switching) behind a C ABI, with boolean circuits (add, mul, matvec)
evaluated level by level and a continuous-batching serving loop.

Importing the package loads nothing; the compiled library is loaded on the
first call into :mod:`paper_2005_01945_gb300.api`, which raises if it is
missing.
"""

__all__ = ["api", "synth"]
