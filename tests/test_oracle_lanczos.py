"""Pins of the oracle's condition-number estimate from CG's coefficients.

`oracle.lanczos_extremes` turns the step lengths alpha_j and coefficients
beta_j of preconditioned CG into the Lanczos tridiagonal of the preconditioned
operator and returns its extreme eigenvalues.  Pinned against:

* closed forms: the Laplacians of a path (eigenvalues 2 - 2 cos(pi k / n)) and
  of a grid (sums of two path spectra), where plain CG run to exhaustion
  recovers both extremes;
* dense eigensolves: with the MSP and exact PEGP preconditioners, the nonzero
  spectrum of B L equals that of the pencil (L_Gt, L_T) or (L_Gt, L_H)
  (B = Pi P M P^T Pi, M = L_T^+ or L_H^+);
* the paper's bound: Section 3.2's spectral equivalence puts every nonzero
  eigenvalue of L_H^+ L_Gt in [1 - rho, 1], and its Tables 1 and 2 show the
  condition number shrinking as mu goes from 0.8 to 1/sqrt(n).

A dropped diagonal term, a transposed alpha/beta index or a missing square
root moves the Ritz values away from these values by far more than the
tolerances used here.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests._helpers import pencil_eigs


def _extremes(res):
    return oracle.lanczos_extremes(res.alphas, res.betas)


def test_plain_cg_on_a_path_recovers_the_closed_form():
    n = 40
    g = gg.path(n, w=np.ones(n - 1))
    res = oracle.solve(g, gg.rhs(n, seed=1), "none", tol=1e-14, maxit=400)
    assert res.restarts == 0 and len(res.betas) == len(res.alphas) - 1
    lo, hi = _extremes(res)
    assert lo == pytest.approx(2 - 2 * np.cos(np.pi / n), rel=1e-9)
    assert hi == pytest.approx(2 - 2 * np.cos(np.pi * (n - 1) / n), rel=1e-12)


def test_plain_cg_on_a_grid_recovers_the_product_spectrum():
    nx, ny = 12, 9
    g = gg.grid2d(nx, ny, weights="uniform", lo=1.0, hi=1.0, seed=1)
    res = oracle.solve(g, gg.rhs(g.n, seed=2), "none", tol=1e-14, maxit=1000)
    lo, hi = _extremes(res)
    lam = lambda k, m: 2 - 2 * np.cos(np.pi * k / m)  # noqa: E731
    assert lo == pytest.approx(lam(1, nx), rel=1e-8)
    assert hi == pytest.approx(lam(nx - 1, nx) + lam(ny - 1, ny), rel=1e-10)


@pytest.mark.parametrize("kind", ["msp", "pegp_exact"])
@pytest.mark.parametrize("mu", [0.3, 0.8])
def test_ritz_extremes_equal_the_dense_pencil(kind, mu):
    g = gg.grid2d(10, 8, weights="uniform", lo=1.0, hi=2.0, seed=3)
    M = oracle.make_preconditioner(kind, g, mu=mu, coarse_max=4, seed=2)
    res = oracle.pcg(M.ops.L, gg.rhs(g.n, seed=4), M, tol=1e-14, maxit=2000)
    lo, hi = _extremes(res)
    Lm = (M.ops.LT if kind == "msp" else M.ops.LH).toarray()
    ev = pencil_eigs(M.ops.LG.toarray(), Lm)
    ev = ev[ev > 1e-9 * ev.max()]
    # Ritz values lie inside the spectrum and, once CG has converged, next
    # to its ends (a cluster at an end may leave its Ritz value a little in)
    assert ev.min() * (1 - 1e-9) <= lo and hi <= ev.max() * (1 + 1e-9)
    assert hi == pytest.approx(ev.max(), rel=1e-3)
    assert lo == pytest.approx(ev.min(), rel=1e-3)


def test_pegp_exact_spectrum_lies_in_the_theorem_interval():
    """lambda(L_H^+ L_Gt) <= 1 for every mu (L_Gt <= L_H, Section 3.2), and the
    condition number falls from mu = 0.8 to mu = 1/sqrt(n) (Tables 1-2)."""
    g = gg.grid2d(32, weights="uniform", lo=1.0, hi=1.0, seed=1)
    b = gg.rhs(g.n, seed=3)
    kappa = {}
    for mu in (0.8, 1 / 32):
        res = oracle.solve(g, b, "pegp_exact", mu=mu, seed=1, tol=1e-13, maxit=500)
        lo, hi = _extremes(res)
        assert 0.0 < lo <= hi <= 1.0 + 1e-10
        kappa[mu] = hi / lo
    assert kappa[1 / 32] < 2.0 < kappa[0.8]
