"""CPU oracle for the boundary-concentrated FMM (arXiv 2112.00864).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or
run anything in this package.  The product path (the CUDA library and its
Python binding) never imports it and shares no code with it.

O1 ``direct``: the discrete operator by its definition, element pair by
element pair, FP64.  O2 ``fmm``: the same operator with the far field by the
truncated Cartesian Taylor expansions of Sec. 3.3 and the passes of
Algorithms 1-3, FP64, on its own octree.

Parity pins (tests/test_oracle_*.py) tie each function to something other than
itself: closed forms, brute-force quadrature, polynomial identities, finite
differences, the Taylor remainder bound (Eq. est:remain:G) and Galerkin
symmetry.  No function here is "parity unpinned".
"""
from .oracle import *  # noqa: F401,F403
