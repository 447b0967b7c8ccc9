"""GB300 direct-SCF Coulomb/exchange (J/K) build (arXiv 2406.11185).

The compute path is the CUDA library ``lib/libadft.so`` (C ABI in
``include/adft.h``); ``adft`` is its Python binding and ``synth`` the seeded
input generator.  Importing the package loads nothing; the binding loads the
library on first use and raises if it is missing.
"""
__all__ = ["adft", "synth", "build"]
