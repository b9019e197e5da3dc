"""FP64 CPU oracle for the sliCQ transform (test infrastructure only).

This package is the slow, obviously-correct reference that the CUDA path is
checked against.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_1210_0084_gb300``) never imports, links or runs
anything here, and nothing here imports the product path; the two share only
the seeded input generators in ``paper_1210_0084_gb300.signals``, which hold
none of the transform's arithmetic.

Every function in :mod:`oracle.slicq_oracle` cites the passage of
Holighaus, Doerfler, Velasco, Grill, "A framework for invertible, real-time
constant-Q transforms" (arXiv:1210.0084) it follows.
"""

from .slicq_oracle import *  # noqa: F401,F403
