"""GB300-native Monte Carlo tensor-network renormalization (arXiv:1710.03757).

The compute path is the CUDA library libmctrg.so (hand-written sm_103a
kernels behind the C ABI in include/mctrg.h); `paper_1710_03757_gb300.mctrg`
is its thin ctypes binding.  Importing this package loads nothing; the
binding loads the library on first use and fails loudly if it is missing.
"""
