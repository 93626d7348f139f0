"""ORACLE -- test infrastructure only.

Expanded-graph operators formed literally from their definitions:

* P^k = P^2_1 P^3_2 ... P^k_{k-1}, the piecewise-constant prolongation from
  level k to level 1 (Section 2.2, Eq. def:P);
* P(mu) = [I, -mu P^2, (-mu)^2 P^3, ..., (-mu)^(l-1) P^l] in R^{n x ntilde}
  (Section 2.2, the composite prolongation);
* L_Gt = P(mu)^T L_G P(mu), the expanded Laplacian (Section 3.1, Eq. def:L_ell);
* H, the positively weighted expanded graph: the subgraph of G~ that keeps the
  edges of positive weight only, i.e. the negative off-diagonal entries of
  L_Gt, with its own diagonal (Section 3.2, Theorem thm:MSP_cond);
* T, the multilevel sparsifier: the edges of H on the top level, the edges
  between each vertex and its aggregate on the next level, and the edges
  inside each aggregate (Section 3.3).  Reading: "edges inside aggregations"
  is taken on every level below the top and "edges between the levels" as the
  vertex-to-parent edges; on two levels this is exactly the paper's wording.

Expanded vertices are numbered level by level: level-k vertex u has index
offsets[k-1] + u, with u its id in the hierarchy (aggregate creation order).

Deciding which entries of L_Gt are zero: the product P(mu)^T L P(mu) is
evaluated in floating point, so an entry that is zero in exact arithmetic can
come out as a few ulps of the terms it sums.  An entry counts as zero when its
magnitude is at most 1e-12 times the same product taken over absolute values,
|P(mu)|^T |L| |P(mu)|, which bounds the sum of the magnitudes of its terms.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .hierarchy import Hierarchy

ZERO_REL = 1e-12


def laplacian(adj: sp.spmatrix) -> sp.csr_matrix:
    """Graph Laplacian D - A of a weighted adjacency (Section 2.1)."""
    adj = sp.csr_matrix(adj)
    return (sp.diags(np.asarray(adj.sum(axis=1)).ravel()) - adj).tocsr()


def level_prolongations(h: Hierarchy) -> list:
    """[P^1 = I, P^2, ..., P^l], each n x n_k (Section 2.2, Eq. def:P)."""
    n = h.sizes[0]
    out = [sp.identity(n, format="csr")]
    for k, agg in enumerate(h.agg):
        nk, nk1 = h.sizes[k], h.sizes[k + 1]
        step = sp.csr_matrix((np.ones(nk), (np.arange(nk), agg)), shape=(nk, nk1))
        out.append((out[-1] @ step).tocsr())
    return out


def composite_prolongation(h: Hierarchy, mu: float) -> sp.csr_matrix:
    """P(mu) = [I, (-mu) P^2, ..., (-mu)^(l-1) P^l]  (n x ntilde)."""
    blocks = [((-mu) ** k) * Pk for k, Pk in enumerate(level_prolongations(h))]
    return sp.hstack(blocks, format="csr")


def _upper_entries(m: sp.spmatrix):
    """Strictly upper entries (row, col, value) of m, sorted by (row, col).
    In canonical CSR (sorted indices, duplicates summed) they already come
    in that order, so they are picked out without sorting."""
    m = sp.csr_matrix(m)
    m.sum_duplicates()                               # canonical: sorted, no duplicates
    rows = np.repeat(np.arange(m.shape[0], dtype=np.int64), np.diff(m.indptr))
    cols = m.indices.astype(np.int64)
    keep = cols > rows
    return rows[keep], cols[keep], m.data[keep]


def _from_upper(nt: int, i, j, wgt) -> sp.csr_matrix:
    """Laplacian D - A of the symmetric graph given by its upper edge list."""
    a = sp.csr_matrix((np.concatenate([wgt, wgt]), (np.concatenate([i, j]), np.concatenate([j, i]))),
                      shape=(nt, nt))
    return laplacian(a)


@dataclass
class ExpandedOperators:
    mu: float
    n: int
    ntilde: int
    levels: int
    offsets: np.ndarray
    level_of: np.ndarray      # level (1-based) of each expanded vertex
    local_of: np.ndarray      # id within its level
    parent_of: np.ndarray     # expanded index of the aggregate on the next level (-1 on top)
    L: sp.csr_matrix          # original Laplacian (n x n)
    Pmu: sp.csr_matrix        # composite prolongation (n x ntilde)
    LG: sp.csr_matrix         # expanded Laplacian P^T L P (ntilde x ntilde)
    LH: sp.csr_matrix         # Laplacian of the positive subgraph H
    LT: sp.csr_matrix         # Laplacian of the multilevel sparsifier T
    H_edges: tuple            # (i, j, weight) with i < j, sorted by (i, j)
    H_scale: np.ndarray       # |P|^T |L| |P| at each H edge: rounding-error scale of its weight
    T_edges: tuple
    neg_edges: tuple          # the dropped edges (i < j) and their (negative) weights


def expanded_operators(h: Hierarchy, mu: float, *, with_LG: bool = True) -> ExpandedOperators:
    sizes = h.sizes
    nt = h.ntilde
    offs = h.offsets
    level_of = np.concatenate([np.full(s, k + 1, dtype=np.int64) for k, s in enumerate(sizes)])
    local_of = np.concatenate([np.arange(s, dtype=np.int64) for s in sizes])
    parent_of = -np.ones(nt, dtype=np.int64)
    for k, agg in enumerate(h.agg):
        parent_of[offs[k]:offs[k + 1]] = offs[k + 1] + agg.astype(np.int64)

    L = laplacian(h.adj[0])
    Pmu = composite_prolongation(h, mu)
    LG = (Pmu.T @ L @ Pmu).tocsr()
    LG.sum_duplicates()
    absP = abs(Pmu)
    M = (absP.T @ abs(L) @ absP).tocsr()
    M.sum_duplicates()

    # off-diagonal upper entries of L_Gt, with the cancellation-aware zero test
    gi, gj, gv = _upper_entries(LG)
    mi, mj, mv = _upper_entries(M)
    mkey = mi * nt + mj
    gkey = gi * nt + gj
    pos = np.searchsorted(mkey, gkey)
    assert np.all(mkey[pos] == gkey), "pattern of L_Gt must lie inside |P|^T|L||P|"
    nonzero = np.abs(gv) > ZERO_REL * mv[pos]
    gi, gj, gv, gscale = gi[nonzero], gj[nonzero], gv[nonzero], mv[pos][nonzero]
    weight = -gv                                      # edge weight = -(off-diagonal entry)
    pos_e = weight > 0
    Hi, Hj, Hw, Hs = gi[pos_e], gj[pos_e], weight[pos_e], gscale[pos_e]
    neg = (gi[~pos_e], gj[~pos_e], weight[~pos_e])
    LH = _from_upper(nt, Hi, Hj, Hw)

    # multilevel sparsifier: top level, intra-aggregate and vertex-to-parent edges
    top = len(sizes)
    li, lj = level_of[Hi], level_of[Hj]
    same = li == lj
    on_top = same & (li == top)
    intra = same & (li < top) & (parent_of[Hi] == parent_of[Hj])
    to_parent = (lj == li + 1) & (parent_of[Hi] == Hj)
    tsel = on_top | intra | to_parent
    Ti, Tj, Tw = Hi[tsel], Hj[tsel], Hw[tsel]
    LT = _from_upper(nt, Ti, Tj, Tw)

    return ExpandedOperators(
        mu=mu, n=sizes[0], ntilde=nt, levels=len(sizes), offsets=offs, level_of=level_of,
        local_of=local_of, parent_of=parent_of, L=L, Pmu=Pmu, LG=LG if with_LG else None,
        LH=LH, LT=LT, H_edges=(Hi, Hj, Hw), H_scale=Hs, T_edges=(Ti, Tj, Tw), neg_edges=neg)
