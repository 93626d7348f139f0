"""ORACLE -- test infrastructure only.

Stretch of the positive subgraph H over the multilevel sparsifier T
(Section 3.3), the quantity that bounds the MSP's condition number:

* path_stretch: the paper's definition.  For each edge (i, j) of H, its
  stretch is w_ij times the sum of 1/w over the edges of a path from i to j in
  T; T is not a tree (a matched pair and its parent form a triangle), so the
  path is not unique, and the paper takes the one of least total weight
  ("lightest edge weight sum").  The stretch of H is the sum over its edges.
* resistance_stretch: the same sum with the effective resistance of T
  between i and j in place of the path's resistance, which equals
  tr(L_T^+ L_H) = ||K_T||_F^2 (L_H is the sum of w_e b_e b_e^T).  By Rayleigh's
  monotonicity it is at most path_stretch, and it bounds kappa(L_T^+ L_H) from
  above, the chain of inequalities Section 3.3 uses.
* hutchinson_samples: z^T L_T^+ L_H z for Rademacher vectors z, whose mean is
  an unbiased estimate of tr(L_T^+ L_H) (Hutchinson 1989).  Entry i of sample
  s is the sign of the SplitMix64 output with counter s * 2^32 + i (negative
  when the top bit is set), i the expanded index level by level in hierarchy
  order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

from .expanded import ExpandedOperators
from .hierarchy import splitmix64
from .solve import _GroundedSolver


def _edges(Lx: sp.spmatrix):
    """(i, j, w) with i < j of a Laplacian's off-diagonal part."""
    A = sp.triu(-sp.csr_matrix(Lx), k=1).tocoo()
    keep = A.data > 0
    return A.row[keep], A.col[keep], A.data[keep]


def path_stretch(ops: ExpandedOperators) -> float:
    """sum over H's edges of w_ij * sum_{path} 1/w, the path in T of least
    total weight (Dijkstra with edge lengths w); dense over sources, for
    small graphs."""
    ti, tj, tw = _edges(ops.LT)
    nt = ops.ntilde
    # two graphs over T's edges: lengths w (to choose the path) and 1/w
    W = sp.csr_matrix((np.r_[tw, tw], (np.r_[ti, tj], np.r_[tj, ti])), shape=(nt, nt))
    R = sp.csr_matrix((np.r_[1 / tw, 1 / tw], (np.r_[ti, tj], np.r_[tj, ti])), shape=(nt, nt))
    hi, hj, hw = _edges(ops.LH)
    total = 0.0
    srcs = np.unique(hi)
    dist, pred = csg.dijkstra(W, directed=False, indices=srcs, return_predecessors=True)
    row_of = {s: r for r, s in enumerate(srcs)}
    for i, j, w in zip(hi, hj, hw):
        r = row_of[i]
        res, v = 0.0, j
        while v != i:
            u = pred[r, v]
            res += R[u, v]
            v = u
        total += w * res
    return float(total)


def resistance_stretch(ops: ExpandedOperators) -> float:
    """tr(L_T^+ L_H) with a dense pseudo-inverse (small graphs)."""
    LT = ops.LT.toarray()
    m = LT.shape[0]
    J = np.full((m, m), 1.0 / m)
    G = np.linalg.inv(LT + J) - J
    return float(np.trace(G @ ops.LH.toarray()))


def edge_resistance_stretch(ops: ExpandedOperators) -> float:
    """sum over H's edges of w_e (e_i - e_j)^T L_T^+ (e_i - e_j), one solve of
    L_T per edge (small graphs)."""
    solve = _GroundedSolver(ops.LT)
    total = 0.0
    for i, j, w in zip(*_edges(ops.LH)):
        b = np.zeros(ops.ntilde)
        b[i], b[j] = 1.0, -1.0
        x = solve(b)
        total += w * (x[i] - x[j])
    return float(total)


def rademacher(seed: int, sample: int, nt: int) -> np.ndarray:
    """Sample `sample` of the Rademacher vectors (see the module docstring)."""
    base = (int(sample) & 0xFFFFFFFF) << 32
    return np.array([-1.0 if splitmix64(seed, base + i) >> 63 else 1.0 for i in range(nt)])


def hutchinson_samples(ops: ExpandedOperators, samples: int, seed: int) -> np.ndarray:
    """z_s^T L_T^+ L_H z_s for s = 0..samples-1 (L_T^+ by a grounded sparse
    solve, mean removed: the minimum-norm solution)."""
    solve = _GroundedSolver(ops.LT)
    out = np.empty(samples)
    for s in range(samples):
        z = rademacher(seed, s, ops.ntilde)
        u = solve(ops.LH @ z)
        out[s] = z @ (u - u.mean())
    return out
