"""FP64 CPU oracle for graph-form ADMM (Fougner & Boyd, "Parameter Selection and
Pre-Conditioning for a Graph Form Solver").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA path (no kernels, headers,
helpers, tables or constants); the only module both sides use is ``workloads``, which
draws the seeded synthetic inputs and holds none of the method's arithmetic.

Everything here is plain, slow and written to be checked against the paper by eye:
NumPy/SciPy FP64 (a library Cholesky, matrix products and an elementwise loop over
base-function codes), with no blocking, fusion or reordering.

Modules
  prox     base proximal operators h (Section 5 library), the parametric prox
           formula of Section 5, function values.
  equil    regularized Sinkhorn-Knopp (Algorithm 2), the Frobenius rescale of
           Section 4.1.2 / Section 5, folding D and E into the function parameters
           (Section 4.1, the pre-conditioned problem Eq. 12).
  project  graph projection: the KKT form of Eq. 9 and the reduced (block
           elimination) updates of Section 3.5, with an FP64 Cholesky factor.
  admm     Algorithm 1 with over-relaxation (Section 3.2), the feasible iterates of
           Section 3.3, residual stopping Eq. 11 with the Section 3.4 tolerances, the
           half-tuple gap, the adaptive penalty of Section 4.3 with the Section 3.2
           rescale of the scaled duals; unscaling of the returned tuple.

Pins (tests/test_oracle_*.py, run with -m "not gpu"): each part is checked against
something other than itself -- brute-force 1-D minimisation and subgradient
membership for every prox, Sinkhorn-Knopp optimality conditions and limits, the
diagonal-Sigma projection formulas of Section 4.1.1, the KKT solve, normal equations,
soft thresholding, critical-lambda zeros, vertex enumeration on tiny LPs, support
enumeration on tiny NNLS, KKT conditions of the converged solution, the dual
feasibility invariant of Section 3.3, the D/E scaling invariance of Section 4.1, a
hand-worked rho sequence for the adaptive penalty, ADMM replayed in unscaled duals for
the rescale, and the Section 3.4 test evaluated outside the oracle on its returned tuples.
No part of the oracle is left unpinned.
"""
from . import prox, equil, project, admm  # noqa: F401
