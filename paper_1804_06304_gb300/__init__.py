"""GB300-native Monte-Carlo snakuscules (arXiv:1804.06304).

The compute path lives in the CUDA library ``libac.so`` behind a C ABI
(``include/ac.h``); ``paper_1804_06304_gb300.ac`` is the thin ctypes binding with
the same names.  ``synth`` holds the seeded synthetic input generators.
"""
