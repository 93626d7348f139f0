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
    # per inner solve, min over its steps of | ||r|| / (inner_tol ||r~||) - 1 |:
    # how close its stopping test came to flipping (a diagnostic, no arithmetic
    # of the method depends on it)
    inner_margin: list = field(default_factory=list)

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
            self.inner_margin.append(np.inf)
            return y
        z = self._T(r)
        p = z.copy()
        rho = r @ z
        margin = np.inf
        while its < self.inner_maxit:
            q = LH @ p
            alpha = rho / (p @ q)
            y += alpha * p
            r -= alpha * q
            its += 1
            nr = np.linalg.norm(r)
            margin = min(margin, abs(nr / (self.inner_tol * nrt) - 1.0))
            if nr <= self.inner_tol * nrt:
                break
            z = self._T(r)
            rho_new = r @ z
            p = z + (rho_new / rho) * p
            rho = rho_new
        self.inner_iters.append(its)
        self.inner_margin.append(margin)
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
    alphas: list = field(default_factory=list)   # step lengths of the first CG run
    betas: list = field(default_factory=list)    # direction coefficients of that run


def pcg(L: sp.spmatrix, b: np.ndarray, M, *, tol=1e-8, maxit=1000, flexible=False,
        deadline=None) -> SolveResult:
    """Preconditioned CG on the singular consistent system L x = Pi b, x_0 = 0.

    beta = r_k^T z_k / r_{k-1}^T z_{k-1} (standard) or, if flexible,
    beta = z_k^T (r_k - r_{k-1}) / r_{k-1}^T z_{k-1} (FCG(1), Notay 2000).
    L is a sparse matrix or any operator whose product is ``L @ v``.
    deadline (a time.perf_counter() value, optional) ends the iteration after
    the first step completed past it (timing runs; not converged)."""
    import time
    L = sp.csr_matrix(L) if sp.issparse(L) else L
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
    alphas, betas = [], []
    while its < maxit:
        q = L @ p
        alpha = rho / (p @ q)
        if restarts == 0:
            alphas.append(alpha)
        x += alpha * p
        r_old = r
        r = r - alpha * q
        its += 1
        rel = np.linalg.norm(r) / nb
        hist.append(rel)
        if deadline is not None and time.perf_counter() > deadline:
            break
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
        if restarts == 0:
            betas.append(beta)
        p = z + beta * p
        rho = rho_new
    x = _project(x)
    relres = np.linalg.norm(bp - L @ x) / nb
    return SolveResult(x, its, converged, relres, hist, restarts, alphas, betas[:len(alphas) - 1])


def fgmres(L: sp.spmatrix, b: np.ndarray, M, *, tol=1e-8, maxit=1000, restart=30) -> SolveResult:
    """Flexible GMRES(m) with right preconditioning (Saad, SIAM J. Sci. Comput.
    14, 1993), the outer Krylov method of the paper's experiments (Section 4),
    on the singular consistent system L x = Pi b from x_0 = 0.

    A cycle starts from the residual r (v_1 = r / ||r||).  Step j applies the
    preconditioner, z_j = M(v_j), multiplies w = L z_j, orthogonalises w
    against v_1..v_j by modified Gram-Schmidt (column j of the Hessenberg
    matrix, h_(j+1,j) = ||w||, v_(j+1) = w / h_(j+1,j)), applies the earlier
    Givens rotations to the column and a new one that zeroes h_(j+1,j); the
    rotated right-hand side's entry j+1 is the residual norm of the least
    squares solution, recorded relative to ||Pi b|| and tested against tol.
    The cycle ends after `restart` steps or on convergence: y solves the
    triangular system, x += Z y, and the next cycle starts from the true
    residual Pi b - L x.  The iteration count is the number of products with
    L inside the cycles; a cycle whose true residual meets tol ends the solve."""
    L = sp.csr_matrix(L) if sp.issparse(L) else L
    bp = _project(np.asarray(b, dtype=np.float64))
    nb = np.linalg.norm(bp)
    x = np.zeros_like(bp)
    hist = []
    if nb == 0.0:
        return SolveResult(x, 0, True, 0.0, hist)
    m = int(restart)
    r = bp.copy()
    its, cycles, converged = 0, 0, False
    while its < maxit:
        beta = np.linalg.norm(r)
        if beta / nb <= tol:
            converged = True
            break
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        for j in range(m):
            z = M(V[j])
            Z.append(z)
            w = L @ z
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / d, H[j + 1, j] / d
            H[j, j], H[j + 1, j] = d, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            rel = abs(g[j + 1]) / nb
            hist.append(rel)
            if rel <= tol or its >= maxit or hn == 0.0:
                break
            V.append(w / hn)
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        for i in range(k):
            x += y[i] * Z[i]
        cycles += 1
        r = bp - L @ x
        if np.linalg.norm(r) / nb <= tol:
            converged = True
            break
    x = _project(x)
    relres = np.linalg.norm(bp - L @ x) / nb
    return SolveResult(x, its, converged, relres, hist, max(cycles - 1, 0))


def lanczos_extremes(alphas, betas):
    """Smallest and largest eigenvalue of the Lanczos tridiagonal T_k that CG's
    coefficients define (Hestenes-Stiefel / Lanczos connection, e.g. Saad,
    Iterative Methods for Sparse Linear Systems, Sec. 6.7.3):
    T[j, j] = 1/alpha_j + beta_(j-1)/alpha_(j-1),  T[j, j+1] = sqrt(beta_j)/alpha_j.
    Its eigenvalues (Ritz values) lie inside the spectrum of the preconditioned
    operator and approach its extremes as k grows.  Dense eigensolve."""
    a = np.asarray(alphas, dtype=np.float64)
    b = np.asarray(betas, dtype=np.float64)[:len(a) - 1]
    k = len(a)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / a[j] + (b[j - 1] / a[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(b[j]) / a[j]
    ev = np.linalg.eigvalsh(T)
    return ev[0], ev[-1]


def solve(g, b, kind="msp", *, mu=0.8, tol=1e-8, maxit=1000, krylov="cg", restart=30,
          **kw) -> SolveResult:
    """Convenience: build the oracle preconditioner for graph g and run PCG
    (krylov="cg") or FGMRES(restart) (krylov="fgmres")."""
    M = make_preconditioner(kind, g, mu=mu, **kw)
    L = M.ops.L if M.ops is not None else _laplacian_of(g)
    if krylov == "fgmres":
        return fgmres(L, b, M, tol=tol, maxit=maxit, restart=restart)
    return pcg(L, b, M, tol=tol, maxit=maxit, flexible=M.flexible)


def _laplacian_of(g):
    from .expanded import laplacian
    return laplacian(sp.csr_matrix((g.w, g.col_idx, g.row_ptr), shape=(g.n, g.n)))
