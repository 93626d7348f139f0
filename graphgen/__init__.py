"""Seeded synthetic graph and right-hand-side generators.

This module is shared input plumbing for the solver library, the oracle, the
tests and the benchmark.  It holds none of the solver's arithmetic: it only
draws random graphs and vectors and returns them as a symmetric CSR triple
``(row_ptr int64[n+1], col_idx int32[nnz], w float64[nnz])`` with sorted
columns, no self-loops, no duplicate entries and strictly positive weights.

Graph families follow the paper's test problems (Section 4: 2D regular
grids, Watts-Strogatz ring graphs, real networks reduced to their largest
connected component with self-loops dropped and edges made undirected) and
the synthetic stand-ins used for the real-world networks (Chung-Lu power-law
graphs, R-MAT graphs, random geometric graphs).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph

__all__ = [
    "Graph", "from_edges", "grid2d", "grid3d", "ring", "watts_strogatz", "path",
    "star", "chung_lu", "rmat", "rgg", "random_connected", "largest_cc",
    "edge_weights", "rhs", "lattice_2x4",
]


class Graph:
    """Undirected weighted graph in symmetric CSR form (both directions stored)."""

    def __init__(self, row_ptr, col_idx, w, name=""):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.name = name

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def adjacency(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.w, self.col_idx, self.row_ptr), shape=(self.n, self.n))

    def edges(self):
        """Upper-triangle edge list (u < v) with weights."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.row_ptr))
        keep = rows < self.col_idx
        return rows[keep], self.col_idx[keep].astype(np.int64), self.w[keep]

    def __repr__(self):
        return f"Graph({self.name!r}, n={self.n}, m={self.m})"


def from_edges(n, u, v, w=None, name="") -> Graph:
    """Build a symmetric CSR graph from an undirected edge list.

    Self-loops are dropped; duplicate edges are merged keeping the first
    weight drawn (the generators never rely on merged weights being summed).
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if w is None:
        w = np.ones(u.shape[0], dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    keep = u != v
    u, v, w = u[keep], v[keep], w[keep]
    lo, hi = np.minimum(u, v), np.maximum(u, v)
    key = lo * n + hi
    _, first = np.unique(key, return_index=True)
    lo, hi, w = lo[first], hi[first], w[first]
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    ww = np.concatenate([w, w])
    order = np.lexsort((cols, rows))
    rows, cols, ww = rows[order], cols[order], ww[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return Graph(row_ptr, cols.astype(np.int32), ww, name)


def edge_weights(m, kind="unit", lo=1.0, hi=2.0, seed=0) -> np.ndarray:
    """Draw ``m`` undirected edge weights.

    kind: "unit" (all 1), "uniform" (U[lo, hi]), "uniform01" (U(0, 1]),
    "loguniform" (10**U[log10 lo, log10 hi]).
    """
    rng = np.random.default_rng(seed)
    if kind == "unit":
        return np.ones(m, dtype=np.float64)
    if kind == "uniform":
        return rng.uniform(lo, hi, size=m)
    if kind == "uniform01":
        return 1.0 - rng.random(size=m)          # (0, 1]
    if kind == "loguniform":
        return 10.0 ** rng.uniform(math.log10(lo), math.log10(hi), size=m)
    raise ValueError(f"unknown weight kind {kind!r}")


def _weighted(n, u, v, weights, lo, hi, seed, name):
    w = edge_weights(len(u), weights, lo, hi, seed)
    return from_edges(n, u, v, w, name)


def grid2d(nx, ny=None, weights="unit", lo=1.0, hi=2.0, seed=0) -> Graph:
    """nx-by-ny 4-neighbour lattice; vertex id = y*nx + x."""
    ny = nx if ny is None else ny
    ids = np.arange(nx * ny, dtype=np.int64).reshape(ny, nx)
    u = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
    v = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
    order = np.lexsort((v, u))
    return _weighted(nx * ny, u[order], v[order], weights, lo, hi, seed, f"grid2d_{nx}x{ny}")


def grid3d(nx, ny=None, nz=None, weights="unit", lo=1.0, hi=2.0, seed=0) -> Graph:
    """nx-by-ny-by-nz 7-point lattice; vertex id = (z*ny + y)*nx + x."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    ids = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    u = np.concatenate([ids[:, :, :-1].ravel(), ids[:, :-1, :].ravel(), ids[:-1, :, :].ravel()])
    v = np.concatenate([ids[:, :, 1:].ravel(), ids[:, 1:, :].ravel(), ids[1:, :, :].ravel()])
    order = np.lexsort((v, u))
    return _weighted(nx * ny * nz, u[order], v[order], weights, lo, hi, seed,
                     f"grid3d_{nx}x{ny}x{nz}")


def ring(n, k=2, weights="unit", lo=1.0, hi=2.0, seed=0) -> Graph:
    """Ring lattice: each vertex joined to its k nearest neighbours on each side
    (mean degree 2k), the Watts-Strogatz graph before rewiring."""
    u = np.repeat(np.arange(n, dtype=np.int64), k)
    v = (u + np.tile(np.arange(1, k + 1, dtype=np.int64), n)) % n
    lo_, hi_ = np.minimum(u, v), np.maximum(u, v)
    order = np.lexsort((hi_, lo_))
    return _weighted(n, lo_[order], hi_[order], weights, lo, hi, seed, f"ring_{n}_k{k}")


def watts_strogatz(n, k=2, beta=None, weights="unit", lo=1.0, hi=2.0, seed=0) -> Graph:
    """Watts-Strogatz small world: ring lattice of mean degree 2k whose edges are
    rewired with probability beta (default 1/sqrt(n)); largest component kept."""
    beta = 1.0 / math.sqrt(n) if beta is None else beta
    rng = np.random.default_rng(seed)
    u = np.repeat(np.arange(n, dtype=np.int64), k)
    v = (u + np.tile(np.arange(1, k + 1, dtype=np.int64), n)) % n
    rewire = rng.random(u.shape[0]) < beta
    v = v.copy()
    v[rewire] = rng.integers(0, n, size=int(rewire.sum()))
    g = _weighted(n, u, v, weights, lo, hi, seed + 1, f"ws_{n}")
    return largest_cc(g)


def path(n, w=None) -> Graph:
    u = np.arange(n - 1)
    return from_edges(n, u, u + 1, w, f"path_{n}")


def star(leaves, w=None) -> Graph:
    u = np.zeros(leaves, dtype=np.int64)
    return from_edges(leaves + 1, u, np.arange(1, leaves + 1), w, f"star_{leaves}")


def lattice_2x4() -> Graph:
    """The unit-weight 2-by-4 lattice of the paper's worked example (Section 3.1):
    top row 0-1-2-3, bottom row 4-5-6-7, vertical edges i -- i+4."""
    u = [0, 1, 2, 4, 5, 6, 0, 1, 2, 3]
    v = [1, 2, 3, 5, 6, 7, 4, 5, 6, 7]
    return from_edges(8, u, v, None, "lattice_2x4")


def largest_cc(g: Graph) -> Graph:
    """Restrict to the largest connected component, relabelling vertices in
    increasing order of their original ids."""
    ncomp, lab = csgraph.connected_components(g.adjacency(), directed=False)
    if ncomp == 1:
        return g
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)
    newid = -np.ones(g.n, dtype=np.int64)
    newid[keep] = np.arange(keep.shape[0])
    u, v, w = g.edges()
    sel = (newid[u] >= 0) & (newid[v] >= 0)
    return from_edges(keep.shape[0], newid[u[sel]], newid[v[sel]], w[sel], g.name + "_lcc")


def chung_lu(n, avg_deg=16.0, gamma=2.5, weights="uniform01", lo=1.0, hi=2.0, seed=0) -> Graph:
    """Chung-Lu power-law graph, largest connected component.

    Expected degrees follow w_i = c * (i + i0)^(-1/(gamma-1)) scaled to mean
    ``avg_deg``.  Edges are drawn by the standard edge-sampling variant: m =
    n*avg_deg/2 endpoint pairs, each endpoint chosen with probability
    proportional to w_i; self-loops are dropped and repeated pairs merged.
    """
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64)
    beta = 1.0 / (gamma - 1.0)
    # offset i0 caps the largest expected degree near sqrt(n * avg_deg)
    i0 = max(1.0, (math.sqrt(avg_deg) * (1.0 - beta) * n ** (beta - 0.5)) ** (1.0 / beta))
    wdeg = (i + i0) ** (-beta)
    wdeg *= avg_deg * n / wdeg.sum()
    prob = wdeg / wdeg.sum()
    m = int(round(n * avg_deg / 2.0))
    cdf = np.cumsum(prob)
    cdf[-1] = 1.0
    u = np.searchsorted(cdf, rng.random(m), side="right")
    v = np.searchsorted(cdf, rng.random(m), side="right")
    perm = rng.permutation(n)                 # hide the degree ordering in the ids
    u, v = perm[u], perm[v]
    w = edge_weights(m, weights, lo, hi, seed + 1)
    return largest_cc(from_edges(n, u, v, w, f"chunglu_{n}_d{avg_deg:g}"))


def rmat(scale, edge_factor=16, a=0.57, b=0.19, c=0.19, weights="unit", lo=1.0, hi=2.0,
         seed=0) -> Graph:
    """R-MAT graph with 2^scale vertices and edge_factor*2^scale directed draws,
    symmetrised, deduplicated, self-loops dropped, largest component kept."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    m = edge_factor * n
    u = np.zeros(m, dtype=np.int64)
    v = np.zeros(m, dtype=np.int64)
    for bit in range(scale):
        r = rng.random(m)
        right = ((r >= a) & (r < a + b)) | (r >= a + b + c)
        down = r >= a + b
        u |= down.astype(np.int64) << bit
        v |= right.astype(np.int64) << bit
    perm = rng.permutation(n)
    u, v = perm[u], perm[v]
    w = edge_weights(m, weights, lo, hi, seed + 1)
    return largest_cc(from_edges(n, u, v, w, f"rmat_s{scale}_ef{edge_factor}"))


def rgg(n, avg_deg=10.0, weights="loguniform", lo=1e-2, hi=1e2, seed=0) -> Graph:
    """Random geometric graph in the unit square, radius sqrt(avg_deg/(pi n)),
    largest connected component."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    radius = math.sqrt(avg_deg / (math.pi * n))
    pairs = cKDTree(pts).query_pairs(radius, output_type="ndarray")
    w = edge_weights(pairs.shape[0], weights, lo, hi, seed + 1)
    return largest_cc(from_edges(n, pairs[:, 0], pairs[:, 1], w, f"rgg_{n}"))


def random_connected(n, extra=2.0, weights="uniform", lo=1.0, hi=2.0, seed=0) -> Graph:
    """Small random connected graph: a random spanning tree plus ~extra*n random edges."""
    rng = np.random.default_rng(seed)
    parent = np.array([rng.integers(0, i) for i in range(1, n)], dtype=np.int64)
    u = np.concatenate([np.arange(1, n), rng.integers(0, n, int(extra * n))])
    v = np.concatenate([parent, rng.integers(0, n, int(extra * n))])
    w = edge_weights(u.shape[0], weights, lo, hi, seed + 1)
    return from_edges(n, u, v, w, f"random_{n}")


def rhs(n, nrhs=1, seed=0) -> np.ndarray:
    """Right-hand sides with i.i.d. N(0,1) entries, shape (n,) or (nrhs, n)."""
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((nrhs, n))
    return b[0] if nrhs == 1 else b
