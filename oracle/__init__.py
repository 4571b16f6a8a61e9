"""FP64 CPU oracle for LINVIEW (arXiv 1403.6968) -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct numpy implementations of what the maintained
programs compute, written from the paper:

* ``powers``    -- matrix powers and sums of powers: re-evaluation (Table 1),
                   the incremental exponential-model rule (Appendix A, with the
                   "old views, updates last" order of Example 3.8), the sums
                   rule derived from the multi-matrix delta rule (Section 3.4),
                   the multiplication counts of Appendix A, and the adjoint
                   through the squaring chain.
* ``iteration`` -- the general form T_{i+1} = A T_i + B (Section 4.3): re-
                   evaluation, the incremental linear model (Appendix B) and
                   the adjoint of L = ||T_k||_F^2.
* ``ols``       -- OLS (Section 4.1): re-evaluation, Sherman-Morrison
                   (Section 3.1), the two-step Sherman-Morrison of Example 3.3
                   and block Woodbury for row-block replacements.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The CUDA product path never calls it and shares no
code with it; the only common module is ``linview_inputs`` (random inputs).

Everything is float64.  numpy's ``@`` (BLAS) and ``numpy.linalg`` routines are
used as library primitives; there is no blocking, fusion or reordering beyond
what each cited rule states.
"""
from . import powers, iteration, ols  # noqa: F401
from .metrics import rel_frob  # noqa: F401
