"""Solve groups: many graphs of uneven size in one launch per PCG phase.

lap_pcg_solve_group merges the graphs block-diagonally and runs every
(graph, column) pair's CG with its own scalars; the preconditioner of each
graph is its own MSP (Section 3.3).  Checked here, through the C ABI:

* every column of every graph meets relative residual 1e-8 (recomputed on
  the host) and agrees with a single solve of that column on the same handle
  within what the two residuals allow;
* column 0 of every graph agrees with the oracle's FP64 PCG: the solution
  within 2e-8 ||Pi b|| in the residual norm, the iteration count within the
  oracle's own spread under rounding-size changes (``_helpers.ITER_SPREAD``,
  +-1 unless recorded there; tests/test_iteration_spread.py);
* mixed precision, plain CG, a second call reusing the workspace, and the
  refusals (PEGP, mixed mu).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.expanded import laplacian

from _helpers import GROUP_GRAPHS, iter_band

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2207_07847_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build_library()
    P.lib()
    P.set_torch_allocator()
    yield
    torch.cuda.synchronize()


@pytest.fixture(scope="module")
def graphs():
    return [(name, make(), k) for name, make, k in GROUP_GRAPHS]


def _rhs(g, idx, k):
    return np.stack([gg.rhs(g.n, seed=100 + 10 * idx + j) for j in range(k)])


def _solve_group(graphs, precision, prec="msp"):
    hs = [P.lap_setup(g, seed=17, mu=0.8, prec=prec, precision=precision, maxit=6000)
          for _, g, _ in graphs]
    grp = P.Group(hs)
    Bs = [torch.as_tensor(_rhs(g, i, k), device="cuda") for i, (_, g, k) in enumerate(graphs)]
    Xs = [torch.full_like(B, np.nan) for B in Bs]
    st, infos = P.lap_pcg_solve_group(grp, Bs, Xs)
    return hs, grp, Bs, Xs, st, infos


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_group_columns_meet_tolerance_and_match_single_solves(graphs, precision):
    hs, grp, Bs, Xs, st, infos = _solve_group(graphs, precision)
    assert st == 0, [i.as_dict() for i in infos if i.status]
    at = 0
    for idx, (name, g, k) in enumerate(graphs):
        L = laplacian(g.adjacency())
        B, X = Bs[idx].cpu().numpy(), Xs[idx].cpu().numpy()
        for j in range(k):
            bp = B[j] - B[j].mean()
            nb = np.linalg.norm(bp)
            rel = np.linalg.norm(bp - L @ X[j]) / nb
            assert rel <= 1e-8, (name, j, rel, infos[at + j].as_dict())
            assert infos[at + j].status == 0 and infos[at + j].relres <= 1e-8
            assert abs(infos[at + j].relres - rel) <= 1e-3 * rel + 1e-15
            assert abs(X[j].mean()) <= 1e-12 * np.abs(X[j]).max()
        # single solves of the first and last column on the same handle
        for j in sorted({0, k - 1}):
            x1 = torch.empty_like(Bs[idx][j])
            single = P.lap_pcg_solve(hs[idx], Bs[idx][j], x1)
            assert single.status == 0
            bp = B[j] - B[j].mean()
            assert np.linalg.norm(L @ (X[j] - x1.cpu().numpy())) <= 2e-8 * np.linalg.norm(bp), (name, j)
        at += k
    grp.close()


def test_group_column_zero_matches_the_oracle(graphs):
    hs, grp, Bs, Xs, st, infos = _solve_group(graphs, "fp64")
    assert st == 0
    at = 0
    for idx, (name, g, k) in enumerate(graphs):
        b = Bs[idx][0].cpu().numpy()
        ref = oracle.solve(g, b, "msp", mu=0.8, seed=17, maxit=6000)
        assert ref.converged
        L = laplacian(g.adjacency())
        bp = b - b.mean()
        x = Xs[idx][0].cpu().numpy()
        assert np.linalg.norm(L @ (x - ref.x)) <= 2e-8 * np.linalg.norm(bp), name
        band = iter_band(("group", name))
        assert abs(infos[at].iterations - ref.iters) <= band, (name, infos[at].iterations, ref.iters, band)
        at += k
    grp.close()


def test_group_plain_cg_and_workspace_reuse():
    gs = [gg.grid2d(30, 20, weights="uniform", lo=1.0, hi=2.0, seed=3), gg.rgg(900, seed=4),
          gg.chung_lu(2000, avg_deg=10, seed=5)]
    hs = [P.lap_setup(g, seed=1, prec="none", maxit=5000) for g in gs]
    grp = P.Group(hs)
    for call in range(2):
        Bs = [torch.as_tensor(_rhs(g, i + 10 * call, 3), device="cuda") for i, g in enumerate(gs)]
        Xs = [torch.empty_like(B) for B in Bs]
        st, infos = P.lap_pcg_solve_group(grp, Bs, Xs)
        assert st == 0, [i.as_dict() for i in infos]
        for g, B, X in zip(gs, Bs, Xs):
            L = laplacian(g.adjacency())
            for j in range(3):
                b = B[j].cpu().numpy()
                bp = b - b.mean()
                assert np.linalg.norm(bp - L @ X[j].cpu().numpy()) <= 1e-8 * np.linalg.norm(bp)
    grp.close()


def test_group_refusals():
    g1 = gg.grid2d(12, weights="uniform", seed=1)
    g2 = gg.grid2d(14, weights="uniform", seed=2)
    h1 = P.lap_setup(g1, seed=1, prec="pegp_inner")
    h2 = P.lap_setup(g2, seed=1, prec="pegp_inner")
    with pytest.raises(P.LapError) as e:
        P.Group([h1, h2])
    assert e.value.status == 12
    h1 = P.lap_setup(g1, seed=1, mu=0.8)
    h2 = P.lap_setup(g2, seed=1, mu=0.5)
    with pytest.raises(P.LapError) as e:
        P.Group([h1, h2])
    assert e.value.status == 1
