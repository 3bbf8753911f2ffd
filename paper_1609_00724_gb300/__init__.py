"""GB300-native QSL / FLL / FLEDGE engine (arXiv:1609.00724 method).

The compute path lives in the CUDA library libqsl.so (csrc/); `qsl` is its
thin ctypes binding. Importing this package does not load the library; the
first call of a `qsl` function does, and fails loudly if it is missing.
"""
