"""ORACLE -- test infrastructure only.

Preconditioned conjugate gradient on L x = b with the paper's preconditioners.

The paper runs a Krylov method on the expanded system L_Gt x~ = P(mu)^T b
(Section 4) preconditioned by M = L_T^+ (MSP, Section 3.3) or M = L_H^+ (PEGP,
Section 3.2), and recovers x = P(mu) x~ (Section 3.1, the equivalence
theorem).  With x~_0 = 0 this is the same iteration as preconditioned CG on
L x = b with the n x n preconditioner

    B = Pi P(mu) M P(mu)^T Pi,      Pi = I - 1 1^T / n,

whose iterates are x_k = Pi P(mu) x~_k; every step below is that iteration.
The paper uses FGMRES; this build uses conjugate gradients, flexible (Notay's
FCG(1) choice of beta) when the preconditioner is an inner iteration.

* MSP:        M = L_T^+, applied as an exact sparse solve of L_T.
* PEGP exact: M = L_H^+, applied as an exact sparse solve of L_H.
* PEGP inner: M ~= L_H^+ by an inner CG on L_H y = r~ preconditioned by L_T^+,
              from y = 0 until ||r~ - L_H y|| <= inner_tol ||r~||.
* none:       B = Pi (plain CG).

Stopping (reading of "relative residual", Section 4): the recurrence residual
satisfies ||r_k|| <= tol ||Pi b||; the true residual ||Pi b - L x_k|| is then
checked and, if it fails, the iteration restarts from the true residual.
The iteration count is the number of products with L inside the loop.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .expanded import ExpandedOperators, expanded_operators
from .hierarchy import build_hierarchy


class _GroundedSolver:
    """x = A^+ b for a connected graph Laplacian A and b with zero sum:
    solve with the last vertex grounded, then remove the mean."""

    def __init__(self, A: sp.spmatrix):
        A = sp.csc_matrix(A)
        self.n = A.shape[0]
        self.lu = spla.splu(A[:-1, :-1].tocsc()) if self.n > 1 else None

    def __call__(self, b: np.ndarray) -> np.ndarray:
        x = np.zeros(self.n)
        if self.lu is not None:
            x[:-1] = self.lu.solve(np.asarray(b[:-1], dtype=np.float64))
        return x - x.mean()


def _project(v):
    return v - v.mean()


@dataclass
class OraclePreconditioner:
    kind: str
    ops: ExpandedOperators | None
    inner_tol: float = 1e-6
    inner_maxit: int = 500
    inner_iters: list = field(default_factory=list)

    def __post_init__(self):
        if self.kind in ("msp", "pegp_inner"):
            self._T = _GroundedSolver(self.ops.LT)
        if self.kind == "pegp_exact":
            self._H = _GroundedSolver(self.ops.LH)

    @property
    def flexible(self) -> bool:
        return self.kind == "pegp_inner"

    def restrict(self, r):
        """r~ = P(mu)^T Pi r."""
        return self.ops.Pmu.T @ _project(r)

    def prolong(self, yt):
        """z = Pi P(mu) y~."""
        return _project(self.ops.Pmu @ yt)

    def apply_tilde(self, rt):
        """M r~ in the expanded space."""
        if self.kind == "msp":
            return self._T(rt)
        if self.kind == "pegp_exact":
            return self._H(rt)
        if self.kind == "pegp_inner":
            return self._inner(rt)
        raise ValueError(self.kind)

    def __call__(self, r):
        if self.kind == "none":
            return _project(r)
        return self.prolong(self.apply_tilde(self.restrict(r)))

    def _inner(self, rt):
        """Inner CG on L_H y = r~ with preconditioner L_T^+, y_0 = 0."""
        LH = self.ops.LH
        y = np.zeros_like(rt)
        r = rt.copy()
        nrt = np.linalg.norm(rt)
        its = 0
        if nrt == 0.0:
            self.inner_iters.append(0)
            return y
        z = self._T(r)
        p = z.copy()
        rho = r @ z
        while its < self.inner_maxit:
            q = LH @ p
            alpha = rho / (p @ q)
            y += alpha * p
            r -= alpha * q
            its += 1
            if np.linalg.norm(r) <= self.inner_tol * nrt:
                break
            z = self._T(r)
            rho_new = r @ z
            p = z + (rho_new / rho) * p
            rho = rho_new
        self.inner_iters.append(its)
        return y


def make_preconditioner(kind, g=None, *, mu=0.8, coarse_max=32, max_levels=0, seed=0,
                        order_random=True, inner_tol=1e-6, inner_maxit=500, hierarchy=None):
    if kind == "none":
        return OraclePreconditioner("none", None)
    h = hierarchy or build_hierarchy(g.row_ptr, g.col_idx, g.w, coarse_max=coarse_max,
                                     max_levels=max_levels, seed=seed, order_random=order_random)
    ops = expanded_operators(h, mu)
    return OraclePreconditioner(kind, ops, inner_tol=inner_tol, inner_maxit=inner_maxit)


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    converged: bool
    relres: float                    # true relative residual at exit
    history: list                    # recurrence relative residual after each iteration
    restarts: int = 0


def pcg(L: sp.spmatrix, b: np.ndarray, M, *, tol=1e-8, maxit=1000, flexible=False) -> SolveResult:
    """Preconditioned CG on the singular consistent system L x = Pi b, x_0 = 0.

    beta = r_k^T z_k / r_{k-1}^T z_{k-1} (standard) or, if flexible,
    beta = z_k^T (r_k - r_{k-1}) / r_{k-1}^T z_{k-1} (FCG(1), Notay 2000)."""
    L = sp.csr_matrix(L)
    bp = _project(np.asarray(b, dtype=np.float64))
    nb = np.linalg.norm(bp)
    x = np.zeros_like(bp)
    hist = []
    if nb == 0.0:
        return SolveResult(x, 0, True, 0.0, hist)
    r = bp.copy()
    z = M(r)
    p = z.copy()
    rho = r @ z
    its, restarts = 0, 0
    converged = False
    while its < maxit:
        q = L @ p
        alpha = rho / (p @ q)
        x += alpha * p
        r_old = r
        r = r - alpha * q
        its += 1
        rel = np.linalg.norm(r) / nb
        hist.append(rel)
        if rel <= tol:
            rt = bp - L @ x
            if np.linalg.norm(rt) / nb <= tol:
                converged = True
                break
            r = rt                                  # restart from the true residual
            z = M(r)
            p = z.copy()
            rho = r @ z
            restarts += 1
            continue
        z = M(r)
        rho_new = r @ z
        beta = (z @ (r - r_old)) / rho if flexible else rho_new / rho
        p = z + beta * p
        rho = rho_new
    x = _project(x)
    relres = np.linalg.norm(bp - L @ x) / nb
    return SolveResult(x, its, converged, relres, hist, restarts)


def solve(g, b, kind="msp", *, mu=0.8, tol=1e-8, maxit=1000, **kw) -> SolveResult:
    """Convenience: build the oracle preconditioner for graph g and run PCG."""
    M = make_preconditioner(kind, g, mu=mu, **kw)
    L = M.ops.L if M.ops is not None else _laplacian_of(g)
    return pcg(L, b, M, tol=tol, maxit=maxit, flexible=M.flexible)


def _laplacian_of(g):
    from .expanded import laplacian
    return laplacian(sp.csr_matrix((g.w, g.col_idx, g.row_ptr), shape=(g.n, g.n)))
