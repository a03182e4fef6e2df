"""GB300-native time-stepper stability analysis (arXiv:1804.03859 hot path).

``nsstab`` is the thin ctypes binding of the C-ABI library ``libnsstab.so``
(declared in ``include/nsstab.h``); ``inputs`` holds the seeded synthetic
input generators.
"""
