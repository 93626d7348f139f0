"""Serving: continuous batching of solve requests through the C ABI.

The central property: a request's result does not depend on what else the
server is doing.  Every column of a batch runs its own CG with reductions
whose order depends only on the batch width and the handle, so a request
solved alone and the same request solved while other requests (on the same
graph and on other graphs) join and leave the batch give the same bits and
the same iteration count.  The results are also checked against the graph's
true residual and against the oracle's solve.
"""
import threading
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle.expanded import laplacian

from _helpers import iter_band

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2207_07847_gb300")

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def lib_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build_library()
    P.lib()
    P.set_torch_allocator()
    yield
    torch.cuda.synchronize()


def _cols(n, k, seed):
    return np.stack([gg.rhs(n, seed=seed + j) for j in range(k)])


def _relres(g, b, x):
    L = laplacian(g.adjacency())
    bp = b - b.mean()
    return np.linalg.norm(bp - L @ x) / np.linalg.norm(bp)


@pytest.fixture(scope="module")
def graphs():
    gs = [gg.grid2d(56, 40, weights="loguniform", lo=1e-2, hi=1e2, seed=2),
          gg.chung_lu(2500, seed=4),
          gg.watts_strogatz(1800, 6, 0.1, seed=8)]
    hs = [P.lap_setup(gs[0], seed=5, maxit=4000),
          P.lap_setup(gs[1], seed=5, maxit=4000),
          P.lap_setup(gs[2], seed=5, maxit=4000, prec="none")]
    return gs, hs


def _solve_alone(server, h, B):
    Bd = torch.as_tensor(B, device="cuda")
    Xd = torch.full_like(Bd, np.nan)
    rid = server.submit(h, Bd, Xd)
    st, info = server.wait(rid, 120.0)
    return st, info, Xd.cpu().numpy()


def test_request_alone_equals_request_in_the_mix(graphs):
    gs, hs = graphs
    S = P.Server(max_slots=16, check_every=4)
    try:
        probes = [_cols(g.n, k, seed=100 + 10 * i) for i, (g, k) in enumerate(zip(gs, (2, 1, 3)))]
        alone = [_solve_alone(S, h, B) for h, B in zip(hs, probes)]
        for (st, info, X), g, B in zip(alone, gs, probes):
            assert st == 0, info.as_dict()
            for j in range(B.shape[0]):
                assert _relres(g, B[j], X[j]) <= TOL

        # the mix: background requests on every graph, submitted in waves, with
        # the probes submitted while the first wave is in flight (they join
        # running batches at an iteration boundary)
        rng = np.random.default_rng(7)
        keep, ids = [], []

        def bg(i, k, seed):
            Bd = torch.as_tensor(_cols(gs[i].n, k, seed), device="cuda")
            Xd = torch.full_like(Bd, np.nan)
            keep.append((i, Bd, Xd))
            ids.append(S.submit(hs[i], Bd, Xd))

        for w in range(6):
            bg(w % 3, int(rng.integers(1, 5)), 1000 + w)
        time.sleep(0.002)
        probe_out = []
        for h, B in zip(hs, probes):
            Bd = torch.as_tensor(B, device="cuda")
            Xd = torch.full_like(Bd, np.nan)
            probe_out.append((Bd, Xd, S.submit(h, Bd, Xd)))
            bg(int(rng.integers(0, 3)), int(rng.integers(1, 4)), 2000 + len(ids))
        for w in range(6):
            bg(w % 3, int(rng.integers(1, 6)), 3000 + w)
        for (Bd, Xd, rid), (st0, info0, X0) in zip(probe_out, alone):
            st, info = S.wait(rid, 120.0)
            assert st == 0, info.as_dict()
            X = Xd.cpu().numpy()
            assert np.array_equal(X, X0), np.abs(X - X0).max()
            assert info.iterations == info0.iterations
            assert info.relres == info0.relres
        for rid, (i, Bd, Xd) in zip(ids, keep):
            st, info = S.wait(rid, 120.0)
            assert st == 0, info.as_dict()
            B, X = Bd.cpu().numpy(), Xd.cpu().numpy()
            for j in range(B.shape[0]):
                assert _relres(gs[i], B[j], X[j]) <= TOL
    finally:
        S.close()


def test_served_solution_matches_oracle(graphs):
    gs, hs = graphs
    S = P.Server(max_slots=8)
    try:
        B = _cols(gs[0].n, 1, seed=55)
        st, info, X = _solve_alone(S, hs[0], B)
        assert st == 0
        ref = oracle.solve(gs[0], B[0], "msp", seed=5)
        L = laplacian(gs[0].adjacency())
        bp = B[0] - B[0].mean()
        assert abs(info.iterations - ref.iters) <= iter_band(("served_grid2d_56x40", "msp"))
        assert np.linalg.norm(L @ (X[0] - ref.x)) <= 2e-8 * np.linalg.norm(bp)
        assert abs(X[0].mean()) <= 1e-12 * np.abs(X[0]).max()
    finally:
        S.close()


def test_admission_by_memory_budget(graphs):
    """A budget that holds one batch at a time: requests for the other graphs
    wait until the resident batch has drained, then run, all correctly."""
    gs, hs = graphs
    big = max(P.lap_get_hierarchy_info(h)["ntilde"] for h in hs)
    budget = 8 * 16 * (8 * big + 2 * big + 64) + 2 * 8 * 2048 * 16 + (1 << 20) + (1 << 16)
    S = P.Server(max_slots=16, hbm_budget_bytes=budget)
    try:
        reqs = []
        for i in (0, 1, 2, 0, 2, 1):
            Bd = torch.as_tensor(_cols(gs[i].n, 2, seed=70 + len(reqs)), device="cuda")
            Xd = torch.empty_like(Bd)
            reqs.append((i, Bd, Xd, S.submit(hs[i], Bd, Xd)))
        for i, Bd, Xd, rid in reqs:
            st, info = S.wait(rid, 120.0)
            assert st == 0, info.as_dict()
            B, X = Bd.cpu().numpy(), Xd.cpu().numpy()
            for j in range(2):
                assert _relres(gs[i], B[j], X[j]) <= TOL
    finally:
        S.close()
    tiny = P.Server(max_slots=16, hbm_budget_bytes=1 << 20)
    try:
        Bd = torch.as_tensor(_cols(gs[0].n, 1, seed=3), device="cuda")
        with pytest.raises(P.LapError) as e:
            tiny.submit(hs[0], Bd, torch.empty_like(Bd))
        assert e.value.status == 11
    finally:
        tiny.close()


def test_cancel_callback_and_errors(graphs):
    gs, hs = graphs
    g = gg.grid3d(40, weights="loguniform", lo=1e-3, hi=1e3, seed=3)
    h = P.lap_setup(g, seed=5, prec="none", maxit=100000, tol=1e-14)
    S = P.Server(max_slots=8, check_every=8)
    done, lock = [], threading.Lock()

    def cb(rid, info):
        with lock:
            done.append((rid, info["status"]))

    try:
        Bd = torch.as_tensor(_cols(g.n, 1, seed=1), device="cuda")
        Xd = torch.empty_like(Bd)
        slow = S.submit(h, Bd, Xd, callback=cb)
        B2 = torch.as_tensor(_cols(gs[0].n, 2, seed=4), device="cuda")
        X2 = torch.empty_like(B2)
        fast = S.submit(hs[0], B2, X2, callback=cb)
        st, info = S.wait(fast, 120.0)
        assert st == 0
        st, _ = S.wait(slow, 0.001)
        assert st == 9                               # still running
        assert S.cancel(slow) == 0
        st, info = S.wait(slow, 120.0)
        assert st == 10 and info.iterations > 0
        assert np.isfinite(Xd.cpu().numpy()).all()
        with lock:
            assert sorted(done) == sorted([(fast, 0), (slow, 10)])
        with pytest.raises(P.LapError):
            Bw = torch.zeros(9, gs[0].n, dtype=torch.float64, device="cuda")
            S.submit(hs[0], Bw, torch.empty_like(Bw))        # 9 columns > width 8
        assert S.wait(fast, 1.0)[0] == 1                     # already waited for
    finally:
        S.close()


def test_latency_under_load(graphs):
    """Many small requests from a submitting thread: all finish, and the
    server reports per-request latency (submission to completion)."""
    gs, hs = graphs
    S = P.Server(max_slots=32, check_every=8)
    try:
        rng = np.random.default_rng(1)
        reqs = []
        for r in range(60):
            i = int(rng.integers(0, 3))
            Bd = torch.as_tensor(_cols(gs[i].n, 1, seed=500 + r), device="cuda")
            Xd = torch.empty_like(Bd)
            reqs.append((i, Bd, Xd, S.submit(hs[i], Bd, Xd)))
        lat = []
        for i, Bd, Xd, rid in reqs:
            st, info = S.wait(rid, 120.0)
            assert st == 0
            lat.append(info.seconds)
            assert _relres(gs[i], Bd.cpu().numpy()[0], Xd.cpu().numpy()[0]) <= TOL
        lat = np.sort(lat)
        assert lat[0] > 0 and np.isfinite(lat).all()
    finally:
        S.close()


def test_true_residual_restart():
    """A tolerance near what FP64 CG can reach on an ill-conditioned grid: a
    column whose recurrence converged while its true residual did not is
    restarted from the true residual, so that a request reported converged
    really is, and the restart count is reported."""
    g = gg.grid3d(20, weights="loguniform", lo=1e-3, hi=1e3, seed=3)
    h = P.lap_setup(g, seed=5, maxit=20000, tol=3e-13)
    S = P.Server(max_slots=8)
    try:
        B = _cols(g.n, 4, seed=21)
        Bd = torch.as_tensor(B, device="cuda")
        Xd = torch.empty_like(Bd)
        st, info = S.wait(S.submit(h, Bd, Xd), 120.0)
        assert st in (0, 7), info.as_dict()
        X = Xd.cpu().numpy()
        worst = max(_relres(g, B[j], X[j]) for j in range(4))
        assert abs(worst - info.relres) <= 1e-3 * worst + 1e-16
        if st == 0:
            assert worst <= 3e-13
        assert 0 <= info.restarts <= 4
    finally:
        S.close()


def test_mixed_precision_requests_alone_and_in_the_mix(graphs):
    """LAP_MIXED handles: FP32 columns refined per request against their FP64
    true residual; converged to 1e-8, the same bits alone and in the mix, and
    close to the oracle's FP64 solve."""
    gs, _ = graphs
    hs = [P.lap_setup(gs[0], seed=5, maxit=4000, precision="mixed"),
          P.lap_setup(gs[1], seed=5, maxit=4000, precision="mixed")]
    S = P.Server(max_slots=16, check_every=4)
    try:
        probe = _cols(gs[0].n, 2, seed=61)
        st0, info0, X0 = _solve_alone(S, hs[0], probe)
        assert st0 == 0, info0.as_dict()
        assert info0.refinements >= 1
        for j in range(2):
            assert _relres(gs[0], probe[j], X0[j]) <= TOL
        keep = []
        for w in range(4):
            i = w % 2
            Bd = torch.as_tensor(_cols(gs[i].n, 1 + w, seed=900 + w), device="cuda")
            Xd = torch.empty_like(Bd)
            keep.append((i, Bd, Xd, S.submit(hs[i], Bd, Xd)))
        Bp = torch.as_tensor(probe, device="cuda")
        Xp = torch.empty_like(Bp)
        rid = S.submit(hs[0], Bp, Xp)
        st, info = S.wait(rid, 120.0)
        assert st == 0
        assert np.array_equal(Xp.cpu().numpy(), X0)
        assert info.iterations == info0.iterations and info.refinements == info0.refinements
        for i, Bd, Xd, r in keep:
            st, info = S.wait(r, 120.0)
            assert st == 0, info.as_dict()
            B, X = Bd.cpu().numpy(), Xd.cpu().numpy()
            for j in range(B.shape[0]):
                assert _relres(gs[i], B[j], X[j]) <= TOL
        ref = oracle.solve(gs[0], probe[0], "msp", seed=5)
        L = laplacian(gs[0].adjacency())
        bp = probe[0] - probe[0].mean()
        assert np.linalg.norm(L @ (X0[0] - ref.x)) <= 2e-8 * np.linalg.norm(bp)
    finally:
        S.close()
