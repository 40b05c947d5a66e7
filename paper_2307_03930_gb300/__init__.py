"""GB300 (sm_103a) row-skipping outer-product SpMM (Rosko, arXiv 2307.03930).

The compute lives in a C-ABI shared library built from ``csrc/`` (see
``include/rosko.h``); ``paper_2307_03930_gb300.rosko`` is its thin ctypes
binding.  ``inputs`` holds the seeded synthetic input generators.
"""
