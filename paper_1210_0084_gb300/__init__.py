"""GB300-native sliCQ: the sliced constant-Q nonstationary Gabor transform.

Forward and inverse sliCQ (Holighaus, Doerfler, Velasco, Grill,
arXiv:1210.0084, Algorithms 3 and 4) as hand-written CUDA kernels for sm_103a
behind a C-ABI library (``include/slicq.h``).  The Python layer here only
marshals arguments: importing :mod:`paper_1210_0084_gb300.slicq` loads the
shared library and fails loudly when it is missing.
"""

__all__ = ["signals"]
