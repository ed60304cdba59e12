"""GB300-native crack-length-controlled phase-field FFT solver (arXiv 2412.17445).

The solver is the C ABI library ``librve.so`` (include/rve.h) built from ``csrc/`` for
sm_103a.  ``binding`` holds the thin ctypes binding with the same entry-point names;
``microstructure`` draws seeded synthetic RVEs.  Importing the package does not load the
library; ``binding.lib()`` does, and fails loudly when it is missing.
"""

__all__ = ["binding", "microstructure", "build"]
