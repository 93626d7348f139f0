"""Pins of the oracle's flexible GMRES (the outer method of the paper's
Section 4), independent of its own code:

* the minimal-residual property by brute force: with a fixed preconditioner B,
  step k of right-preconditioned GMRES minimises ||r_0 - L B y|| over the
  Krylov space K_k(L B, r_0); an explicit Krylov basis and a library least
  squares solve give that minimum on tiny graphs;
* finite termination: unrestarted GMRES on an n-vertex graph reaches the
  exact solution in at most n - 1 steps;
* monotone residuals within a cycle, and the converged solution (restarted
  every few steps) equal to the dense pseudo-inverse solution.

A dropped rotation, a transposed Hessenberg index or a wrong back-substitution
breaks the first pin at the first few steps.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.expanded import laplacian


def _dense_solution(g, b):
    L = laplacian(g.adjacency()).toarray()
    J = np.full(L.shape, 1.0 / g.n)
    return (np.linalg.inv(L + J) - J) @ (b - b.mean())


@pytest.mark.parametrize("kind", ["none", "msp", "pegp_exact"])
def test_residuals_are_the_krylov_least_squares_minimum(kind):
    g = gg.random_connected(24, extra=1.5, weights="uniform", seed=7)
    b = gg.rhs(g.n, seed=8)
    M = oracle.make_preconditioner(kind, g, mu=0.5, coarse_max=3, seed=4)
    L = (M.ops.L if M.ops is not None else laplacian(g.adjacency())).toarray()
    res = oracle.fgmres(L, b, M, tol=1e-14, maxit=8, restart=50)
    r0 = b - b.mean()
    nb = np.linalg.norm(r0)
    # B as a dense matrix (it is linear and fixed for these preconditioners)
    B = np.column_stack([M(e) for e in np.eye(g.n)])
    K = [r0 / nb]
    for k in range(1, 7):
        A = L @ B @ np.column_stack(K)
        c, *_ = np.linalg.lstsq(A, r0, rcond=None)
        best = np.linalg.norm(r0 - A @ c) / nb
        assert res.history[k - 1] == pytest.approx(best, rel=1e-7, abs=1e-13)
        v = L @ B @ K[-1]
        for u in K:                                  # keep the basis well conditioned
            v = v - (u @ v) * u
        K.append(v / np.linalg.norm(v))


def test_unrestarted_gmres_terminates_within_n_minus_one_steps():
    n = 10
    g = gg.path(n, w=np.linspace(1.0, 2.0, n - 1))
    b = gg.rhs(n, seed=3)
    res = oracle.solve(g, b, "none", krylov="fgmres", restart=50, tol=1e-12, maxit=50)
    assert res.converged and res.iters <= n - 1
    np.testing.assert_allclose(res.x, _dense_solution(g, b), atol=1e-10 * np.abs(res.x).max())


@pytest.mark.parametrize("kind,restart", [("none", 7), ("msp", 5), ("pegp_exact", 30),
                                          ("pegp_inner", 10)])
def test_restarted_solution_equals_the_dense_solve(kind, restart):
    g = gg.grid2d(12, weights="uniform", lo=1.0, hi=2.0, seed=1)
    b = gg.rhs(g.n, seed=2)
    res = oracle.solve(g, b, kind, mu=0.8, coarse_max=4, seed=1, krylov="fgmres",
                       restart=restart, tol=1e-12, maxit=3000, inner_tol=1e-13)
    assert res.converged
    xs = _dense_solution(g, b)
    assert np.linalg.norm(res.x - xs) <= 1e-9 * np.linalg.norm(xs)
    # within a cycle the least squares residual never grows
    h = np.asarray(res.history)
    cyc = [h[i:i + restart] for i in range(0, len(h), restart)]
    for c in cyc:
        assert np.all(np.diff(c) <= 1e-12 * c[0])


def test_restart_one_is_the_minimal_residual_iteration():
    """FGMRES(1) takes, each step, the multiple of z = M(r) that minimises the
    residual: x += a z with a = (r, L z) / (L z, L z), then r = Pi b - L x."""
    g = gg.grid2d(7, 5, weights="uniform", lo=1.0, hi=2.0, seed=2)
    b = gg.rhs(g.n, seed=6)
    M = oracle.make_preconditioner("msp", g, mu=0.8, coarse_max=4, seed=1)
    L = M.ops.L
    res = oracle.fgmres(L, b, M, tol=1e-30, maxit=15, restart=1)
    bp = b - b.mean()
    x = np.zeros(g.n)
    for k in range(15):
        r = bp - L @ x
        z = M(r)
        q = L @ z
        x = x + (r @ q) / (q @ q) * z
        rel = np.linalg.norm(bp - L @ x) / np.linalg.norm(bp)
        assert res.history[k] == pytest.approx(rel, rel=1e-9)
    np.testing.assert_allclose(res.x, x - x.mean(), atol=1e-12 * np.abs(x).max())
