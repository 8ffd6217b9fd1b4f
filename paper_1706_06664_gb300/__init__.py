"""GB300-native ACE hot path: SRP hashing, count-array insert, gather score, threshold.

The compute lives in ``csrc/`` (hand-written CUDA for sm_103a behind the C ABI declared in
``include/ace.h``); ``ace.py`` is the ctypes binding.  Importing this package does not load
the CUDA library; the first binding call does, and fails loudly if it is missing.
"""
