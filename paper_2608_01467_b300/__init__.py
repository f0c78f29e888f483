"""feynsparse on B300: reduced Feynman-history amplitudes (arxiv 2608.01467).

The compute path is libfeynsparse.so (C ABI in include/feynsparse.h, CUDA
kernels for sm_103a).  This package is the thin binding over it; importing
it does not load the library, the first call does (and fails loudly when the
library has not been built).
"""
from .api import Batch, Circuit, amplitudes, gates_to_abi  # noqa: F401
