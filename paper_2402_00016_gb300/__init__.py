"""GB300-native Multipolynomial Monte Carlo trace estimation.

The compute path is libmmc.so (hand-written CUDA for sm_103a behind the C
ABI of include/mmc.h); ``paper_2402_00016_gb300.mmc`` is its ctypes binding.
Importing this package does not load the library; ``from
paper_2402_00016_gb300 import mmc`` does, and fails loudly if it is missing.
"""
