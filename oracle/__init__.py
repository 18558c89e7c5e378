"""Slow, plain FP64 CPU oracle of the non-planar spectral BIEM time step.

TEST INFRASTRUCTURE ONLY: this package exists to check the CUDA path.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the product package
``paper_2107_03550_gb300``; the two meet only through the seeded input
generators in ``paper_2107_03550_gb300.workloads``, which hold none of the
method's arithmetic.

Modules:
  kernels -- W, C^T_II, C^N_II (Sec. 2.3, Sec. 2.4, App. A)
  sbiem   -- windows, weights, friction Newton, the two-pass step (Sec. 3)

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, the elastodynamic Laplace-domain responses, invariants or
brute force; none is "parity unpinned".
"""
from .kernels import G_N, G_T, W  # noqa: F401
from .sbiem import Oracle, Params, newton_lnV, state_update, weights, windows  # noqa: F401
