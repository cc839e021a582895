"""GB300-native FastFCA: joint-diagonalisation-based multichannel Wiener filtering.

The compute path lives in the CUDA library ``libfastfca.so`` built from ``csrc/``; the
binding in ``fastfca.py`` marshals arguments to its C ABI (``include/fastfca.h``).
Importing this package does not load the library; ``fastfca`` does, and raises if it
has not been built.
"""
