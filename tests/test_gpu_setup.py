"""Setup on the device (setup_device = 1): the handshake-matching hierarchy
(Section 2.2, its data-parallel variant) and PEGP's L_H (Section 3.2) built
by device kernels.

Checked bit for bit against the host build of the same options (every level's
aggregates and pairs, T's edges, which carry the coarse weights and the
out-weights, and H's edges with their weights) and against the oracle's
plain-loop hierarchy and expanded operators; then solves on a device-built
and a host-built handle give identical residual histories, which also covers
the degrees and L_H's diagonal."""
import numpy as np
import pytest

import graphgen as gg
import oracle
import paper_2207_07847_gb300 as P

pytestmark = pytest.mark.gpu


def _shuffled_rows(g, seed):
    """The same graph with every row's entries in a random order (the coarse
    weights are summed in CSR order, so the order is part of the input)."""
    rng = np.random.default_rng(seed)
    ci, w = g.col_idx.copy(), g.w.copy()
    for u in range(g.n):
        a, b = g.row_ptr[u], g.row_ptr[u + 1]
        p = rng.permutation(b - a) + a
        ci[a:b], w[a:b] = ci[p], w[p]
    return g.row_ptr, ci, w


GRAPHS = [
    ("grid2d", lambda: gg.grid2d(64, weights="uniform", lo=1, hi=2, seed=1)),
    ("grid3d", lambda: gg.grid3d(14, 13, 12, weights="loguniform", lo=1e-3, hi=1e3, seed=3)),
    ("chunglu", lambda: gg.chung_lu(3000, avg_deg=16, seed=4)),
    ("rmat", lambda: gg.rmat(11, 16, seed=5)),
    ("rgg", lambda: gg.rgg(2500, seed=6)),
    ("path", lambda: gg.path(4097)),
    ("star", lambda: gg.star(600)),
    ("grid2d_unit", lambda: gg.grid2d(40, 37)),
]


def _csr(g):
    return (g.row_ptr, g.col_idx, g.w) if hasattr(g, "row_ptr") else g


def _outputs(h):
    info = P.lap_get_hierarchy_info(h)
    aggs = [P.lap_get_aggregates(h, k + 1) for k in range(info["levels"] - 1)]
    return info, aggs, P.lap_get_expanded_edges(h, 1), P.lap_get_expanded_edges(h, 0)


def _same_bits(a, b):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape
    if a.dtype == np.float64:
        assert np.array_equal(a.view(np.int64), b.view(np.int64))
    else:
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name,make", GRAPHS, ids=[g[0] for g in GRAPHS])
@pytest.mark.parametrize("shuffle", [False, True], ids=["sorted", "shuffled"])
def test_device_setup_bit_exact_with_host_and_oracle(name, make, shuffle):
    g = make()
    rp, ci, w = _shuffled_rows(g, 17) if shuffle else _csr(g)
    kw = dict(matching="handshake", prec="pegp_inner", mu=0.8)
    hd = P.lap_setup(rp, ci, w, setup_device=1, **kw)
    hh = P.lap_setup(rp, ci, w, host_only=1, **kw)
    dinfo, daggs, dT, dH = _outputs(hd)
    hinfo, haggs, hT, hH = _outputs(hh)
    assert dinfo["level_size"] == hinfo["level_size"]
    assert dinfo["nnz_H"] == hinfo["nnz_H"] and dinfo["edges_T"] == hinfo["edges_T"]
    for a, b in zip(daggs, haggs):
        for x, y in zip(a, b):
            _same_bits(x, y)
    for a, b in zip(dT + dH, hT + hH):
        _same_bits(a, b)
    # the oracle's plain loops: aggregates, pairs, and the edge sets of T and H
    ho = oracle.build_hierarchy(rp, ci, w, matching="handshake")
    assert dinfo["level_size"] == ho.sizes
    for k in range(ho.levels - 1):
        agg, pa, pb = daggs[k]
        np.testing.assert_array_equal(agg, ho.agg[k])
        np.testing.assert_array_equal(pa, ho.pair_a[k])
        np.testing.assert_array_equal(pb, ho.pair_b[k])
    if g.n <= 5000:
        # the oracle forms the weights from sparse products of signed entries
        # (a different rounding order with cancellation: 2.3e-10 relative on
        # the log-uniform grid), so its weights agree to 1e-9, the host's bit
        # for bit
        ops = oracle.expanded_operators(ho, 0.8, with_LG=False)
        for got, ref in ((dT, ops.T_edges), (dH, ops.H_edges)):
            np.testing.assert_array_equal(got[0], ref[0])
            np.testing.assert_array_equal(got[1], ref[1])
            np.testing.assert_allclose(got[2], ref[2], rtol=1e-9, atol=0)
    hd.close()
    hh.close()


@pytest.mark.parametrize("prec", ["msp", "pegp_inner"])
def test_device_setup_solves_like_the_host_setup(prec):
    """Identical models give identical solves: FP64 residual histories equal
    bit for bit (the matvec kernel is fixed so that no timing choice enters)."""
    import torch

    g = gg.grid3d(24, 23, 22, weights="loguniform", lo=1e-3, hi=1e3, seed=3)
    kw = dict(matching="handshake", prec=prec, mu=0.8, spmv_tpr=-1, tol=1e-8, maxit=3000,
              inner_tol=0.1, inner_maxit=12)
    hd = P.lap_setup(g, setup_device=1, **kw)
    hg = P.lap_setup(g, setup_device=0, **kw)
    b = torch.as_tensor(gg.rhs(g.n, seed=41), device="cuda")
    x1, x2 = torch.empty_like(b), torch.empty_like(b)
    i1 = P.lap_pcg_solve(hd, b, x1)
    i2 = P.lap_pcg_solve(hg, b, x2)
    assert i1.status == 0 and i2.status == 0
    assert i1.iterations == i2.iterations and i1.inner_iterations == i2.inner_iterations
    _same_bits(P.lap_get_history(hd), P.lap_get_history(hg))
    assert torch.equal(x1, x2)
    hd.close()
    hg.close()


def test_device_setup_larger_graph_matches_host():
    """A grid with about 110,000 vertices (several radix-sort tiles per level
    and many matching rounds): hierarchy and H equal the host build's."""
    g = gg.grid3d(48, weights="loguniform", lo=1e-3, hi=1e3, seed=3)
    kw = dict(matching="handshake", prec="pegp_inner", mu=0.8)
    hd = P.lap_setup(g, setup_device=1, **kw)
    hh = P.lap_setup(g, host_only=1, **kw)
    dinfo, daggs, dT, dH = _outputs(hd)
    hinfo, haggs, hT, hH = _outputs(hh)
    assert dinfo["level_size"] == hinfo["level_size"]
    for a, b in zip(daggs, haggs):
        for x, y in zip(a, b):
            _same_bits(x, y)
    for a, b in zip(dT + dH, hT + hH):
        _same_bits(a, b)
    hd.close()
    hh.close()
