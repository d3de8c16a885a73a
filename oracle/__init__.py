"""CPU FP64 oracle for Tensor Train Multiplication (arXiv:2410.19747).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it. It shares no code with the
CUDA path (``paper_2410_19747_gb300``) and imports nothing from it.

Everything here is plain numpy / LAPACK in float64, written to be checked by
eye against the paper:

* ``tt``      -- tensor-train basics: dense contraction (brute force), the exact
                 Kronecker-core product of Sec. II.A (Eq. carriageXi), inner
                 products / norms through two- and three-layer environments,
                 and dense gradients of the two product functionals.
* ``ttm``     -- the paper's TTM algorithm (Sec. II.B, Eq. tensor, Eq. contract,
                 Eq. eps, Fig. 1): concatenation, Contract, Swap with SVD
                 truncation, QR gauge moves; plus TT-SVD rounding used by the
                 conventional route (Kronecker cores, then rounding).

Parity status of each function is stated in its docstring ("pinned by ..." or
"parity unpinned").
"""

from . import tt, ttm  # noqa: F401
