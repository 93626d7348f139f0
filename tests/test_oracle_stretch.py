"""Pins of the oracle's stretch of H over the sparsifier T (Section 3.3):

* the inequality chain the paper uses, kappa(L_T^+ L_H) <= ||K_T||_F^2 =
  tr(L_T^+ L_H) <= stretch_T(H), with kappa from a dense eigensolve and the
  eigenvalues of L_T^+ L_H at least 1 on its range (T is a subgraph of H);
* the trace computed two independent ways (a dense pseudo-inverse, and one
  sparse solve per edge summing w_e times the effective resistance);
* the lightest path by brute force: on a tiny expanded graph every simple
  path between the ends of each edge is enumerated;
* Hutchinson's estimator: each sample equals z^T L_T^+ L_H z formed densely,
  the Rademacher entries follow the stated SplitMix64 counters, and the mean
  over many samples lies within four standard errors of the trace.
"""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import stretch
from tests._helpers import pencil_eigs


def _ops(g, mu, coarse_max=4, seed=2):
    h = oracle.build_hierarchy(g.row_ptr, g.col_idx, g.w, coarse_max=coarse_max, seed=seed)
    return oracle.expanded_operators(h, mu)


@pytest.mark.parametrize("mu", [0.3, 0.8])
def test_stretch_chain_of_inequalities(mu):
    g = gg.grid2d(9, 7, weights="uniform", lo=1.0, hi=2.0, seed=3)
    ops = _ops(g, mu)
    ev = pencil_eigs(ops.LH.toarray(), ops.LT.toarray())
    ev = ev[ev > 1e-9 * ev.max()]
    assert ev.min() >= 1.0 - 1e-9
    tr = stretch.resistance_stretch(ops)
    assert tr == pytest.approx(ev.sum(), rel=1e-9)
    assert ev.max() / ev.min() <= tr
    assert tr == pytest.approx(stretch.edge_resistance_stretch(ops), rel=1e-9)
    assert tr <= stretch.path_stretch(ops) * (1 + 1e-12)


def test_lightest_path_by_brute_force():
    g = gg.path(6, w=np.array([1.0, 3.0, 2.0, 5.0, 1.5]))
    ops = _ops(g, 0.5, coarse_max=2, seed=1)
    ti, tj, tw = stretch._edges(ops.LT)
    adj = {}
    for a, b, w in zip(ti, tj, tw):
        adj.setdefault(a, {})[b] = w
        adj.setdefault(b, {})[a] = w
    nt = ops.ntilde
    assert nt <= 12

    def lightest(i, j):
        best = None
        others = [v for v in range(nt) if v not in (i, j)]
        for r in range(len(others) + 1):
            for mid in itertools.permutations(others, r):
                p = (i,) + mid + (j,)
                if all(p[t + 1] in adj.get(p[t], {}) for t in range(len(p) - 1)):
                    cost = sum(adj[p[t]][p[t + 1]] for t in range(len(p) - 1))
                    res = sum(1.0 / adj[p[t]][p[t + 1]] for t in range(len(p) - 1))
                    if best is None or cost < best[0]:
                        best = (cost, res)
        return best[1]

    want = sum(w * lightest(i, j) for i, j, w in zip(*stretch._edges(ops.LH)))
    assert stretch.path_stretch(ops) == pytest.approx(want, rel=1e-12)


def test_rademacher_counters_and_hutchinson():
    g = gg.grid2d(8, 6, weights="uniform", lo=1.0, hi=2.0, seed=5)
    ops = _ops(g, 0.8)
    z = stretch.rademacher(7, 3, ops.ntilde)
    for i in (0, 1, ops.ntilde - 1):
        bit = oracle.splitmix64(7, (3 << 32) + i) >> 63
        assert z[i] == (-1.0 if bit else 1.0)
    vals = stretch.hutchinson_samples(ops, 400, seed=7)
    LT = ops.LT.toarray()
    m = LT.shape[0]
    J = np.full((m, m), 1.0 / m)
    M = (np.linalg.inv(LT + J) - J) @ ops.LH.toarray()
    for s in (0, 17, 399):
        zs = stretch.rademacher(7, s, m)
        assert vals[s] == pytest.approx(zs @ M @ zs, rel=1e-9)
    tr = np.trace(M)
    assert abs(vals.mean() - tr) <= 4 * vals.std() / np.sqrt(len(vals))
