"""FP64 CPU oracle of the ALM-BM hot path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import anything from this package.  The product path (the CUDA
library and its Python binding) never imports it and shares no code with it.

Every function is plain, slow, FP64 numpy/scipy, written from the paper:
see ``oracle.alm`` for the per-function citations.  ``oracle.gnn`` is the FP64 reference
of the learned warm start (a network the paper does not have; its definition is stated
there), pinned by ``tests/test_oracle_gnn.py`` (published SplitMix64 outputs, adjoint of
the aggregation, finite differences of the loss, closed-form loss of the zero network).

Parity status
-------------
All functions are pinned by tests in ``tests/test_oracle_*.py`` against closed
forms, the paper's worked examples (``tests/golden/``), finite differences,
interpolation, brute force and dense eigendecompositions.  One part is
*parity unpinned*: nothing fixes the iteration counts of ``solve`` (the paper
prints none), only its end results (objective values and KKT residuals).
"""
from .alm import (  # noqa: F401
    OracleProblem, amap, cost, adjoint, slack_sparse, slack_matvec, slack_dense, precondition,
    aug_lagrangian, dual_candidate, gradient, quartic_coeffs, quartic_value,
    exact_step, lanczos_min, lambda_min, growth_step, kkt, solve, SolveOptions,
    block_growth_map, block_growth_step, psd_sqrt, lbfgs_direction,
)
