"""GB300-native thermal pseudopotential MRT lattice Boltzmann step (arXiv 2206.00946).

The compute path is the C-ABI library ``liblbm.so`` (hand-written sm_103a CUDA,
declared in include/lbm.h); ``paper_2206_00946_gb300.lbm`` is its thin ctypes
binding.  Importing this package does not load the library.
"""
