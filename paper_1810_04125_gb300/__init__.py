"""GB300 (sm_103a) library for adaptive randomized HSS compression
(arXiv:1810.04125): hand-written CUDA kernels behind the C ABI of
include/hss.h, with a thin ctypes binding in ``hss``."""
