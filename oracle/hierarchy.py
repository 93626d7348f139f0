"""ORACLE -- test infrastructure only.

The aggregation hierarchy of Section 2.2: repeated maximal-weight matching
coarsening with Galerkin coarse graphs, until the coarsest level has at most
``coarse_max`` vertices (the paper's "level = max" runs stop at two top
vertices, Section 3.2 before Table 1) or ``max_levels`` levels exist (the
paper's "level = 2" runs, Tables 3-4).  A level with fewer than two aggregates
is never created.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import _cbuild


def splitmix64(seed: int, i: int) -> int:
    """i-th output of SplitMix64 (Steele, Lea & Flood, 2014) started at seed."""
    return int(_cbuild.lib().oh_splitmix64(seed & (2**64 - 1), i & (2**64 - 1)))


@dataclass
class Hierarchy:
    """Levels 1..l of the aggregation hierarchy (stored 0-based: index k-1).

    adj[k]    weighted adjacency of level k+1 (symmetric CSR, zero diagonal)
    agg[k]    aggregate id at level k+2 of each level-(k+1) vertex (len l-1)
    pair_a[k], pair_b[k]  the matched pair that created each aggregate
    """
    adj: list = field(default_factory=list)
    agg: list = field(default_factory=list)
    pair_a: list = field(default_factory=list)
    pair_b: list = field(default_factory=list)

    @property
    def levels(self) -> int:
        return len(self.adj)

    @property
    def sizes(self) -> list:
        return [a.shape[0] for a in self.adj]

    @property
    def ntilde(self) -> int:
        return int(sum(self.sizes))

    @property
    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)


def _match(adj: sp.csr_matrix, seed: int, level: int, randomise: bool):
    L = _cbuild.lib()
    n = adj.shape[0]
    rp = np.ascontiguousarray(adj.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(adj.indices, dtype=np.int32)
    w = np.ascontiguousarray(adj.data, dtype=np.float64)
    agg = np.empty(n, dtype=np.int32)
    pa = np.empty(max(n, 1), dtype=np.int32)
    pb = np.empty(max(n, 1), dtype=np.int32)
    nc = L.oh_match(n, rp.ctypes.data, ci.ctypes.data, w.ctypes.data, seed & (2**64 - 1),
                    level, 1 if randomise else 0, agg.ctypes.data, pa.ctypes.data, pb.ctypes.data)
    return agg, int(nc), pa[:nc].copy(), pb[:nc].copy()


def _heaviest(adj: sp.csr_matrix, u: int, eligible) -> int:
    """Heaviest neighbour v of u with eligible[v]; ties to the smaller id; -1 if none."""
    best, best_w = -1, 0.0
    for p in range(adj.indptr[u], adj.indptr[u + 1]):
        v = int(adj.indices[p])
        if not eligible[v]:
            continue
        wv = float(adj.data[p])
        if best < 0 or wv > best_w or (wv == best_w and v < best):
            best, best_w = v, wv
    return best


def _match_handshake(adj: sp.csr_matrix):
    """Deterministic parallel matching (a method change against the paper's
    random-order greedy pass, for data-parallel setup): in rounds, every
    unmatched vertex points at its heaviest unmatched neighbour (ties to the
    smaller id), and two vertices that point at each other are matched; the
    rounds stop when no unmatched vertex has an unmatched neighbour (each round
    matches at least the pair at the heaviest remaining edge, so they end).
    Pairs are numbered by their smaller end, ascending, with pair_a the smaller
    end; a leftover joins the aggregate of its heaviest neighbour, which is
    matched.  Plain loops: test sizes only."""
    n = adj.shape[0]
    mate = np.full(n, -1, dtype=np.int64)
    while True:
        free = mate < 0
        cand = np.array([_heaviest(adj, u, free) if free[u] else -1 for u in range(n)])
        mutual = [u for u in range(n) if cand[u] >= 0 and cand[cand[u]] == u]
        if not mutual:
            break
        for u in mutual:
            mate[u] = cand[u]
    agg = np.full(n, -1, dtype=np.int32)
    pa, pb = [], []
    for u in range(n):
        if mate[u] > u:
            agg[u] = agg[mate[u]] = len(pa)
            pa.append(u)
            pb.append(int(mate[u]))
    everyone = np.ones(n, dtype=bool)
    for u in range(n):
        if agg[u] < 0:
            agg[u] = agg[_heaviest(adj, u, everyone)]
    return agg, len(pa), np.array(pa, dtype=np.int32), np.array(pb, dtype=np.int32)


def _coarse(adj: sp.csr_matrix, agg: np.ndarray, nc: int) -> sp.csr_matrix:
    L = _cbuild.lib()
    n = adj.shape[0]
    rp = np.ascontiguousarray(adj.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(adj.indices, dtype=np.int32)
    w = np.ascontiguousarray(adj.data, dtype=np.float64)
    nnz = L.oh_coarse(n, rp.ctypes.data, ci.ctypes.data, w.ctypes.data, agg.ctypes.data, nc,
                      None, None, None)
    crp = np.empty(nc + 1, dtype=np.int64)
    cci = np.empty(max(nnz, 1), dtype=np.int32)
    cw = np.empty(max(nnz, 1), dtype=np.float64)
    L.oh_coarse(n, rp.ctypes.data, ci.ctypes.data, w.ctypes.data, agg.ctypes.data, nc,
                crp.ctypes.data, cci.ctypes.data, cw.ctypes.data)
    m = sp.csr_matrix((cw[:nnz], cci[:nnz], crp), shape=(nc, nc))
    m.has_sorted_indices = True
    return m


def build_hierarchy(row_ptr, col_idx, w, *, coarse_max: int = 32, max_levels: int = 0,
                    seed: int = 0, order_random: bool = True,
                    matching: str = "greedy") -> Hierarchy:
    """Aggregation hierarchy of the graph given as symmetric CSR (no self-loops).

    matching="greedy" is the paper's pass (Section 2.2, vertices in random
    order); "handshake" the deterministic parallel variant (_match_handshake;
    seed and order_random unused).  The input rows are used in the order given
    (their CSR order fixes the order in which level-2 weights are summed)."""
    n = len(row_ptr) - 1
    adj = sp.csr_matrix((np.asarray(w, dtype=np.float64), np.asarray(col_idx, dtype=np.int32),
                         np.asarray(row_ptr, dtype=np.int64)), shape=(n, n))
    h = Hierarchy(adj=[adj])
    k = 1
    while True:
        cur = h.adj[-1]
        if cur.shape[0] <= coarse_max:
            break
        if max_levels and k >= max_levels:
            break
        if matching == "handshake":
            agg, nc, pa, pb = _match_handshake(cur)
        else:
            agg, nc, pa, pb = _match(cur, seed, k, order_random)
        if nc < 2:
            break
        h.agg.append(agg)
        h.pair_a.append(pa)
        h.pair_b.append(pb)
        h.adj.append(_coarse(cur, agg, nc))
        k += 1
    return h
