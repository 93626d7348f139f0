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
