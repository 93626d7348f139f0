"""Host-side logic of the solver library, checked without a GPU.

The library's setup stage (validation, matching hierarchy, sparsifier T and
PEGP H construction) runs on the host; with ``host_only=1`` it touches no GPU,
so its integer outputs can be compared bit-for-bit with the oracle here.
"""
import re

import numpy as np
import pytest

import graphgen as gg
import oracle

P = pytest.importorskip("paper_2207_07847_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2207_07847_gb300 import build
    build.build()
    P.lib()


def _declared_functions():
    with open(P.os.path.join(P.os.path.dirname(P._HERE), "include", "lap.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lap_[a-z_]+)\s*\(", src)) - {"lap_alloc_fn", "lap_free_fn",
                                                                   "lap_done_cb"})


def test_library_exports_every_declared_function():
    names = _declared_functions()
    assert len(names) >= 20
    lib = P.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert {s[0] for s in P.SIGNATURES} == set(names)


def test_options_defaults_and_status_strings():
    o = P.make_options()
    assert o.prec == 1 and o.precision == 0 and o.mu == 0.8 and o.coarse_max == 32
    assert o.tol == 1e-8 and o.maxit == 1000
    for s in range(13):
        assert P.lib().lap_status_string(s)


GRAPHS = [
    ("grid2d", lambda: gg.grid2d(64, weights="uniform", lo=1, hi=2, seed=1)),
    ("grid3d", lambda: gg.grid3d(14, 13, 12, weights="loguniform", lo=1e-3, hi=1e3, seed=3)),
    ("chunglu", lambda: gg.chung_lu(3000, avg_deg=16, seed=4)),
    ("rmat", lambda: gg.rmat(11, 16, seed=5)),
    ("rgg", lambda: gg.rgg(2500, seed=6)),
    ("ws", lambda: gg.watts_strogatz(1024, seed=2)),
]


@pytest.mark.parametrize("name,make", GRAPHS, ids=[g[0] for g in GRAPHS])
@pytest.mark.parametrize("seed,order_random,coarse_max", [(7, 1, 32), (0, 0, 2), (123, 1, 5)])
def test_hierarchy_bit_exact_with_oracle(name, make, seed, order_random, coarse_max):
    g = make()
    h = P.lap_setup(g, host_only=1, seed=seed, order_random=order_random, coarse_max=coarse_max)
    ho = oracle.build_hierarchy(g.row_ptr, g.col_idx, g.w, coarse_max=coarse_max, seed=seed,
                                order_random=bool(order_random))
    info = P.lap_get_hierarchy_info(h)
    assert info["level_size"] == ho.sizes
    assert info["ntilde"] == ho.ntilde
    for k in range(ho.levels - 1):
        agg, pa, pb = P.lap_get_aggregates(h, k + 1)
        np.testing.assert_array_equal(agg, ho.agg[k])
        np.testing.assert_array_equal(pa, ho.pair_a[k])
        np.testing.assert_array_equal(pb, ho.pair_b[k])


@pytest.mark.parametrize("name,make", GRAPHS[:4], ids=[g[0] for g in GRAPHS[:4]])
@pytest.mark.parametrize("mu", [0.8, 0.3])
def test_sparsifier_and_pegp_edges_bit_exact(name, make, mu):
    g = make()
    h = P.lap_setup(g, host_only=1, seed=11, mu=mu, prec="pegp_inner")
    ho = oracle.build_hierarchy(g.row_ptr, g.col_idx, g.w, seed=11)
    ops = oracle.expanded_operators(ho, mu, with_LG=False)
    # The oracle forms each weight as a sum of signed terms (P^T L P); its rounding
    # error is bounded by a few ulps of |P|^T |L| |P| at that entry (H_scale).
    Hscale = dict(zip(zip(ops.H_edges[0].tolist(), ops.H_edges[1].tolist()), ops.H_scale))
    for which, ref in ((1, ops.T_edges), (0, ops.H_edges)):
        i, j, w = P.lap_get_expanded_edges(h, which)
        np.testing.assert_array_equal(i, ref[0])
        np.testing.assert_array_equal(j, ref[1])
        scale = np.array([Hscale[(a, b)] for a, b in zip(i.tolist(), j.tolist())])
        assert np.all(np.abs(w - ref[2]) <= 1e-13 * np.abs(ref[2]) + 1e-12 * scale)
    assert P.lap_get_hierarchy_info(h)["edges_T"] == len(ops.T_edges[0])


def test_threaded_setup_equals_single_threaded_and_oracle(monkeypatch):
    """Setup splits its large loops (coarse graphs, H's edges and rows, the
    SELL layout) over host threads; every output is produced by one thread in
    the sequential order, so one thread and many give the same bits, and the
    oracle's integer outputs."""
    g = gg.grid3d(24, weights="loguniform", lo=1e-3, hi=1e3, seed=3)
    outs = []
    for threads in ("1", "8"):
        monkeypatch.setenv("LAP_SETUP_THREADS", threads)
        h = P.lap_setup(g, host_only=1, seed=11, mu=0.8, prec="pegp_inner")
        info = P.lap_get_hierarchy_info(h)
        got = [P.lap_get_expanded_edges(h, which) for which in (0, 1)]
        got += [P.lap_get_aggregates(h, k + 1) for k in range(info["levels"] - 1)]
        outs.append(got)
    for a, b in zip(outs[0], outs[1]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    ho = oracle.build_hierarchy(g.row_ptr, g.col_idx, g.w, seed=11)
    ops = oracle.expanded_operators(ho, 0.8, with_LG=False)
    i, j, w = outs[1][0]
    np.testing.assert_array_equal(i, ops.H_edges[0])
    np.testing.assert_array_equal(j, ops.H_edges[1])
    for k in range(ho.levels - 1):
        np.testing.assert_array_equal(outs[1][2 + k][0], ho.agg[k])


@pytest.mark.parametrize("name,make", GRAPHS, ids=[g[0] for g in GRAPHS])
def test_handshake_matching_bit_exact_with_oracle(name, make):
    """The deterministic parallel matching variant: aggregates and pairs of
    every level, H's and T's edges, equal to the oracle's plain-loop version;
    each level's matching is maximal (no two adjacent unmatched vertices) and
    its pairs are edges."""
    g = make()
    h = P.lap_setup(g, host_only=1, matching="handshake", prec="pegp_inner", mu=0.8)
    ho = oracle.build_hierarchy(g.row_ptr, g.col_idx, g.w, matching="handshake")
    info = P.lap_get_hierarchy_info(h)
    assert info["level_size"] == ho.sizes
    for k in range(ho.levels - 1):
        agg, pa, pb = P.lap_get_aggregates(h, k + 1)
        np.testing.assert_array_equal(agg, ho.agg[k])
        np.testing.assert_array_equal(pa, ho.pair_a[k])
        np.testing.assert_array_equal(pb, ho.pair_b[k])
        adj = ho.adj[k].tocsr()
        assert np.all(adj[pa, pb] > 0)
        matched = np.zeros(adj.shape[0], dtype=bool)
        matched[pa] = matched[pb] = True
        free = np.flatnonzero(~matched)
        assert adj[free][:, free].nnz == 0
    if name in ("grid2d", "rgg"):
        ops = oracle.expanded_operators(ho, 0.8, with_LG=False)
        for which, ref in ((1, ops.T_edges), (0, ops.H_edges)):
            i, j, w = P.lap_get_expanded_edges(h, which)
            np.testing.assert_array_equal(i, ref[0])
            np.testing.assert_array_equal(j, ref[1])


def test_handshake_matching_threads_and_options(monkeypatch):
    g = gg.grid3d(24, weights="loguniform", lo=1e-3, hi=1e3, seed=3)
    outs = []
    for threads in ("1", "8"):
        monkeypatch.setenv("LAP_SETUP_THREADS", threads)
        h = P.lap_setup(g, host_only=1, matching="handshake", seed=5)
        info = P.lap_get_hierarchy_info(h)
        outs.append([P.lap_get_aggregates(h, k + 1) for k in range(info["levels"] - 1)])
    for a, b in zip(outs[0], outs[1]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    # the seed does not enter the variant
    h2 = P.lap_setup(g, host_only=1, matching="handshake", seed=99)
    for k, ref in enumerate(outs[0]):
        assert np.array_equal(P.lap_get_aggregates(h2, k + 1)[0], ref[0])
    assert P.lap_setup_status(g.row_ptr, g.col_idx, g.w, matching=2, host_only=1) == 1


def test_library_reproduces_table_level_sizes():
    for n in (16, 64, 256, 1024):
        s = int(round(n ** 0.5))
        for g in (gg.grid2d(s), gg.ring(n, 2)):
            h = P.lap_setup(g, host_only=1, order_random=0, coarse_max=2)
            info = P.lap_get_hierarchy_info(h)
            assert info["level_size"] == [n >> k for k in range(info["levels"])]


def _status(rp, ci, w, **kw):
    return P.lap_setup_status(rp, ci, w, host_only=1, **kw)


def test_validation_rejects_bad_input():
    g = gg.grid2d(4)
    rp, ci, w = g.row_ptr.copy(), g.col_idx.copy(), g.w.copy()
    assert _status(rp, ci, w) == 0
    w2 = w.copy()
    w2[0] = 2.0
    assert _status(rp, ci, w2) == 2                   # weight asymmetry
    w3 = w.copy()
    w3[3] = -1.0
    assert _status(rp, ci, w3) == 4                   # bad weight
    w4 = w.copy()
    w4[5] = np.nan
    assert _status(rp, ci, w4) == 4
    ci2 = ci.copy()
    ci2[0] = 0                                        # self-loop at vertex 0
    assert _status(rp, ci2, w) == 1
    ci3 = ci.copy()
    ci3[1] = ci3[0]                                   # duplicate entry
    assert _status(rp, ci3, w) == 1
    ci4 = ci.copy()
    ci4[0] = 99                                       # out of range
    assert _status(rp, ci4, w) == 1
    two = gg.from_edges(4, [0, 2], [1, 3])            # two components
    assert _status(two.row_ptr, two.col_idx, two.w) == 3
    assert _status(np.array([0]), np.array([], np.int32), np.array([])) == 1   # n = 0
    assert _status(rp, ci, w, mu=1.5) == 1
    assert _status(rp, ci, w, tol=0.0) == 1


@pytest.mark.parametrize("threads", ["1", "8"])
def test_validation_of_large_graphs_on_threads(monkeypatch, threads):
    """Validation splits its row passes over host threads on large inputs:
    each error is still found, and when a graph has several the one reported
    is the one a sequential scan meets first (entry errors before duplicates
    before asymmetry; the smallest row within a pass)."""
    monkeypatch.setenv("LAP_SETUP_THREADS", threads)
    g = gg.grid3d(32, weights="uniform", lo=1.0, hi=2.0, seed=1)
    rp, ci, w = g.row_ptr.copy(), g.col_idx.copy(), g.w.copy()
    assert rp[-1] > 1 << 16                            # the threaded path
    assert _status(rp, ci, w) == 0
    late = rp[g.n - 5]                                 # an entry of a late row
    w2 = w.copy()
    w2[late] *= 1.5
    assert _status(rp, ci, w2) == 2                    # asymmetry
    w3 = w2.copy()
    w3[late + 1] = -1.0
    assert _status(rp, ci, w3) == 4                    # bad weight reported before asymmetry
    ci2 = ci.copy()
    ci2[late] = ci2[late + 1]                          # duplicate (and then asymmetry)
    assert _status(rp, ci2, w) == 1
    ci3 = ci.copy()
    ci3[rp[g.n // 2]] = g.n // 2                       # self-loop in a middle row
    w4 = w.copy()
    w4[rp[g.n - 3]] = np.inf                           # and a bad weight later
    assert _status(rp, ci3, w4) == 1
    w5 = w.copy()
    w5[rp[10]] = 0.0                                   # bad weight in an early row wins
    assert _status(rp, ci3, w5) == 4


def test_setup_takes_a_scipy_adjacency():
    g = gg.grid2d(20, 15, weights="uniform", seed=4)
    A = g.adjacency()
    h1 = P.lap_setup(g, host_only=1, seed=2)
    h2 = P.lap_setup(A.tocoo(), host_only=1, seed=2)
    assert P.lap_get_hierarchy_info(h1)["level_size"] == P.lap_get_hierarchy_info(h2)["level_size"]
    np.testing.assert_array_equal(P.lap_get_aggregates(h1, 1)[0], P.lap_get_aggregates(h2, 1)[0])


def test_single_level_when_graph_is_small():
    g = gg.path(5, w=[1.0, 2.0, 3.0, 4.0])
    h = P.lap_setup(g, host_only=1)
    assert P.lap_get_hierarchy_info(h)["levels"] == 1


def test_host_only_handle_refuses_device_work():
    g = gg.grid2d(8)
    h = P.lap_setup(g, host_only=1)
    assert P.lib().lap_pcg_solve(h, 8, 16, None, None) == 1


def test_device_setup_option_validation():
    """setup_device needs the handshake matching; host_only ignores it (the
    host build runs); other values are rejected."""
    g = gg.grid2d(12)
    assert P.lap_setup_status(g.row_ptr, g.col_idx, g.w, setup_device=1, matching="greedy") == 1
    assert P.lap_setup_status(g.row_ptr, g.col_idx, g.w, setup_device=2, matching="handshake",
                              host_only=1) == 1
    h = P.lap_setup(g, setup_device=1, matching="handshake", host_only=1, prec="pegp_inner")
    ref = P.lap_setup(g, matching="handshake", host_only=1, prec="pegp_inner")
    for which in (0, 1):
        for a, b in zip(P.lap_get_expanded_edges(h, which), P.lap_get_expanded_edges(ref, which)):
            assert np.array_equal(a, b)
