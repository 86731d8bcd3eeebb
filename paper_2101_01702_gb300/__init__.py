"""GB300 (sm_103a) implementation of the fused reactive-mixture lattice
Boltzmann step of arXiv 2101.01702.

The compiled library lives in _build/liblbm.so (see build.py); lbm.py binds
its C ABI (include/lbm.h).  Import `paper_2101_01702_gb300.lbm` to use it.
"""
