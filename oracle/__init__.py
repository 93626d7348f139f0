"""ORACLE -- test infrastructure only.

A plain, slow, FP64 CPU restatement of what the solver computes, written from
the paper (Hu & Lin, "Solving Graph Laplacians via Multilevel Sparsifiers"):

* ``oracle.hierarchy``  -- the matching-based aggregation hierarchy (Section 2.2),
  sequential C in ``hier.c`` plus a thin ctypes wrapper, and the deterministic
  parallel matching variant in plain loops;
* ``oracle.expanded``   -- the composite prolongation P(mu) (Section 2.2), the
  expanded Laplacian P(mu)^T L P(mu) (Eq. def:L_ell, Section 3.1), the
  positively-weighted expanded graph H (Section 3.2) and the multilevel
  sparsifier T (Section 3.3), each formed literally as sparse matrices;
* ``oracle.solve``      -- the preconditioners z = P(mu) M P(mu)^T r with
  M = L_T^+ (MSP) or L_H^+ (PEGP, exact or by an inner iteration), the outer
  preconditioned conjugate gradient iteration, flexible GMRES, and the extreme
  eigenvalues of CG's Lanczos tridiagonal;
* ``oracle.stretch``    -- the stretch of H over T (Section 3.3): the path
  stretch, its effective-resistance form tr(L_T^+ L_H) and Hutchinson samples.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library (``paper_2207_07847_gb300``) and the library never imports it; the
two meet only through the seeded input generators in ``graphgen``.

Parity pins for every function live in ``tests/test_oracle_*.py``.  Functions
without an independent pin say "parity unpinned" in their docstring.
"""
from .hierarchy import Hierarchy, build_hierarchy, splitmix64  # noqa: F401
from .expanded import ExpandedOperators, expanded_operators, laplacian  # noqa: F401
from .solve import (  # noqa: F401
    OraclePreconditioner, fgmres, lanczos_extremes, make_preconditioner, pcg, SolveResult,
    solve,
)
