"""Test-only helpers: dense spectral quantities and golden-file readers."""
import os

import numpy as np

import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_symbolic_matrix(name, mu):
    """Read a golden matrix whose entries are Python expressions in mu."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(eval(tok, {"__builtins__": {}}, {"mu": mu})) for tok in line.split()])
    return np.array(rows)


def read_table(name):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


def pencil_eigs(A, B, rel=1e-10):
    """Eigenvalues of the pencil A v = lam B v on range(B) for symmetric PSD B
    (congruence with an orthonormal basis of range(B), then Cholesky)."""
    A = np.asarray(A, dtype=float)
    B = np.asarray(B, dtype=float)
    w, V = np.linalg.eigh(B)
    Q = V[:, w > rel * w.max()]
    Bs = Q.T @ B @ Q
    As = Q.T @ A @ Q
    C = np.linalg.cholesky((Bs + Bs.T) / 2)
    Ci = np.linalg.inv(C)
    return np.linalg.eigvalsh(Ci @ ((As + As.T) / 2) @ Ci.T)


def kappa_nonzero(A, B, zero=1e-9):
    """lambda_max / smallest nonzero lambda of the pencil (A, B) on range(B)."""
    ev = pencil_eigs(A, B)
    evp = ev[ev > zero]
    return evp.max() / evp.min()


# The graphs of the GPU parity cases (tests/test_gpu_parity.py), also used by
# the CPU test of the oracle's rounding spread.
PARITY_GRAPHS = {
    "grid2d_64": lambda: gg.grid2d(64, weights="uniform", lo=1.0, hi=2.0, seed=1),
    "grid3d_20": lambda: gg.grid3d(20, 19, 18, weights="loguniform", lo=1e-3, hi=1e3, seed=3),
    "chunglu_4k": lambda: gg.chung_lu(4096, avg_deg=16, seed=4),
    "rmat_11": lambda: gg.rmat(11, 16, seed=5),
    "rgg_3k": lambda: gg.rgg(3000, seed=6),
}


# The graphs of the GPU group-solve test (tests/test_gpu_group.py): uneven
# sizes from 1.5e2 to 1e5 vertices, several families, each with its own
# number of right-hand sides; the right-hand sides of graph g are
# gg.rhs(n, seed=100 + 10 g + j), j < nrhs.
GROUP_GRAPHS = [
    ("path_150", lambda: gg.path(150, w=np.linspace(1, 3, 149)), 3),
    ("grid2d_20x17", lambda: gg.grid2d(20, 17, weights="uniform", lo=1.0, hi=2.0, seed=11), 1),
    ("rgg_1200", lambda: gg.rgg(1200, seed=12), 5),
    ("chunglu_3000", lambda: gg.chung_lu(3000, avg_deg=12, seed=13), 16),
    ("grid3d_16x15x14", lambda: gg.grid3d(16, 15, 14, weights="loguniform", lo=1e-3, hi=1e3, seed=14), 2),
    ("ring_9000", lambda: gg.ring(9000, 2, weights="uniform", seed=15), 7),
    ("grid2d_160x150", lambda: gg.grid2d(160, 150, weights="loguniform", lo=1e-2, hi=1e2, seed=16), 4),
    ("rmat_14", lambda: gg.rmat(14, 16, seed=17), 9),
    ("grid3d_40", lambda: gg.grid3d(40, weights="uniform", lo=1.0, hi=2.0, seed=18), 1),
    ("grid2d_320x310", lambda: gg.grid2d(320, 310, weights="uniform", lo=1.0, hi=2.0, seed=19), 3),
]


def hub_graph():
    """Six hubs in a path, each with its own leaves (2,500, 2,500, 8,000,
    8,000, 300 and 300): every hub's aggregate holds all its leaves, so the
    sweeps meet aggregates of thousands of members (eliminated by a warp) and
    subtrees too large for shared memory (run in global memory)."""
    sizes = [2500, 2500, 8000, 8000, 300, 300]
    u, v = [], []
    nxt = len(sizes)
    for hb, k in enumerate(sizes):
        u += [hb] * k
        v += list(range(nxt, nxt + k))
        nxt += k
    u += list(range(len(sizes) - 1))
    v += list(range(1, len(sizes)))
    w = gg.edge_weights(len(u), "loguniform", 1e-2, 1e2, seed=7)
    return gg.from_edges(nxt, np.array(u), np.array(v), w, "hubs")


# Iteration-count bands of the FP64 GPU parity cases.  The target is +-1.
# The GPU evaluates every product in another order than the oracle and solves
# the sparsifier by elimination instead of a pivoted sparse LU; both are
# accurate FP64 evaluations, and the preconditioner's output is fixed only to
# within the forward error of an FP64 solve of L_T (or L_H), which grows with
# their conditioning.  CG turns such differences into whole iterations on
# badly conditioned systems.  tests/test_iteration_spread.py runs the oracle
# against itself with only that freedom used -- matvecs summed in reverse
# entry order, other fill-reducing orderings of the factorisations, random
# perturbations of each matvec element by its typical rounding error and of each
# preconditioner output by twice its own FP64 refinement correction -- and
# checks that its count spreads by exactly the band recorded here, or by at
# most 1 for every case left at +-1.
ITER_SPREAD = {
    ("grid3d_20", "msp"): 16,
    ("grid3d_20", "none"): 15,
    ("rgg_3k", "msp"): 2,
    ("rgg_3k", "none"): 2,
    ("hubs", "msp"): 2,
    ("ragged_path", 1000): 7,
    ("ragged_ring", 1000): 8,
    ("ragged_path", 4097): 19,
    ("ragged_ring", 4097): 18,
    # columns 0 and 5 of the batched 18 x 17 x 16 grid (batched vs single)
    ("batched_grid3d_18", "msp", 0): 8,
    ("batched_grid3d_18", "msp", 5): 10,
    ("batched_grid3d_18", "none", 0): 14,
    ("batched_grid3d_18", "none", 5): 9,
    ("served_grid2d_56x40", "msp"): 7,
    # column 0 of the group-solve graphs
    ("group", "grid3d_16x15x14"): 8,
    ("group", "ring_9000"): 6,
    ("group", "grid2d_160x150"): 16,
    ("group", "grid3d_40"): 2,
    ("group", "grid2d_320x310"): 5,
}


def iter_band(key):
    """Allowed |iterations(GPU) - iterations(oracle)| for a parity case."""
    return max(1, ITER_SPREAD.get(key, 1))


def reversed_csr(A):
    """The same sparse matrix with every row's entries stored in reverse
    order, so that a matvec sums them in the other order."""
    import scipy.sparse as sp
    A = sp.csr_matrix(A)
    rp = A.indptr.copy()
    ci = A.indices.copy()
    v = A.data.copy()
    for i in range(A.shape[0]):
        a, b = rp[i], rp[i + 1]
        ci[a:b] = ci[a:b][::-1]
        v[a:b] = v[a:b][::-1]
    B = sp.csr_matrix((v, ci, rp), shape=A.shape)
    B.has_sorted_indices = False
    return B


class GroundedLU:
    """A^+ b for a connected Laplacian A by sparse LU of A with its last
    vertex grounded, under a chosen fill-reducing column ordering."""

    def __init__(self, A, permc_spec):
        import scipy.sparse as sp
        import scipy.sparse.linalg as spla
        A = sp.csc_matrix(A)
        self.n = A.shape[0]
        self.lu = spla.splu(A[:-1, :-1].tocsc(), permc_spec=permc_spec)

    def __call__(self, b):
        x = np.zeros(self.n)
        x[:-1] = self.lu.solve(np.asarray(b[:-1], dtype=np.float64))
        return x - x.mean()


EPS64 = 2.0 ** -53


class RoundedProduct:
    """The sparse matrix A whose products A @ p have every element moved by a
    random multiple in [-1, 1] of the typical rounding error of an FP64 sum
    of k terms, sqrt(k) x 2^-53 x (|A| |p|)_i (k the row length): another
    valid evaluation order's result."""

    def __init__(self, A, seed):
        import scipy.sparse as sp
        self.A = sp.csr_matrix(A)
        self.absA = abs(self.A)
        self.k = np.sqrt(np.diff(self.A.indptr)) * EPS64
        self.rng = np.random.default_rng(seed)
        self.shape = self.A.shape

    def __matmul__(self, p):
        q = self.A @ p
        return q + self.rng.uniform(-1.0, 1.0, q.size) * self.k * (self.absA @ np.abs(p))


class PerturbedSolve:
    """A Laplacian solver whose every output y = solve(b) moves by a random
    zero-sum vector of norm 2 ||d||, where d = solve(b - A y) is the
    correction one FP64 refinement step would make: that correction is the
    size of this solve's forward error, and another FP64 solve of the same
    system (another elimination order) may differ from this one by the sum
    of both forward errors."""

    def __init__(self, solve, A, seed, scale=2.0):
        import scipy.sparse as sp
        self.solve, self.A, self.scale = solve, sp.csr_matrix(A), scale
        self.rng = np.random.default_rng(seed)

    def __call__(self, b):
        y = self.solve(b)
        res = b - self.A @ y
        res -= res.mean()
        d = self.solve(res)
        g = self.rng.standard_normal(y.size)
        g -= g.mean()
        y = y + self.scale * np.linalg.norm(d) * g / np.linalg.norm(g)
        return y - y.mean()
