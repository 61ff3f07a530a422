"""GB300 (sm_103a) atlas packer: the data-parallel hot path of TABI
(Gu, Vining, Sheffer, arXiv 2602.07782) behind the C ABI of include/tabi.h.

``tabi`` is the ctypes binding; ``build`` compiles the CUDA library."""
