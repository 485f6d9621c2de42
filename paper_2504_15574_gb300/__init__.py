"""GB300-native vielbein lattice Boltzmann on the sphere (arXiv 2504.15574).

The numerics run in hand-written CUDA kernels for sm_103a inside ``libvlbm.so``
(sources in ``csrc/``), reached through a C ABI (``include/vlbm.h``).  The Python
layer only marshals arguments; importing this package does not load the library
(``paper_2504_15574_gb300.vlbm`` does, and fails loudly if it is missing).
"""
__all__ = ["inputs"]
