"""GB300-native sliCQ: the sliced constant-Q nonstationary Gabor transform.

Forward and inverse sliCQ (Holighaus, Doerfler, Velasco, Grill,
arXiv:1210.0084, Algorithms 3 and 4) as hand-written CUDA kernels for sm_103a
behind a C-ABI library (``include/slicq.h``).  The Python layer here only
marshals arguments: the first plan, batch or stream of
:mod:`paper_1210_0084_gb300.slicq` (or its ``load_library()``) loads the
shared library and raises OSError when it has not been built; there is no
fallback.
"""

__all__ = ["signals"]
