"""The allocation-free residual entry point, checked against the existing ones.

``lap_laplacian_residual_noalloc`` serves callers that cannot allocate device
memory (a process whose device-memory quota is spent, such as an
out-of-memory handler reporting on its last iterate, or code that must not
touch an allocator it shares): it takes the graph and vectors as device
arrays and keeps its reduction scratch in a fixed array inside the library.
Its output must equal what the regular entry points give: r = Pi b - L x
with L x from ``lap_laplacian_apply``, on two calls in a row (the second call
reuses the scratch the first one left), and repeated calls must leave the
device's free memory unchanged.

The file name sorts last, so pytest collects it after every other test file:
if it fails, a run that stops at the first failure (``-x``) has already run
all the other tests.  It also passes alone in a fresh process (its first call
then does the one-time lookup of the scratch array's address).
"""
import numpy as np
import pytest

import graphgen as gg

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2207_07847_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.build_library()
    P.lib()
    yield
    torch.cuda.synchronize()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dtype)


def test_noalloc_residual_matches_regular_entry_points():
    g = gg.grid3d(24, 23, 21, weights="loguniform", lo=1e-3, hi=1e3, seed=3)
    rp = _dev(g.row_ptr, torch.int64)
    ci = _dev(g.col_idx, torch.int32)
    w = _dev(g.w)
    h = P.lap_setup(g, seed=1)
    for call, seed in enumerate((11, 12)):               # two calls in a row
        x = _dev(gg.rhs(g.n, seed=seed))
        b = _dev(gg.rhs(g.n, seed=seed + 100) + 0.5)      # nonzero mean on purpose
        y = torch.empty_like(x)
        P.lap_laplacian_apply(h, x, y)                    # existing entry point: L x
        torch.cuda.synchronize()
        want = (b - b.mean()) - y
        r = torch.empty_like(x)
        st, rnorm, bnorm = P.lap_laplacian_residual_noalloc(rp, ci, w, x, b, r)
        assert st == 0, (call, st)
        scale = (torch.abs(b) + 2 * torch.abs(x) * g.w.max() * 6).max().item()
        assert torch.max(torch.abs(r - want)).item() <= 1e-13 * scale
        assert abs(rnorm - torch.linalg.norm(want).item()) <= 1e-12 * torch.linalg.norm(want).item()
        assert abs(bnorm - torch.linalg.norm(b - b.mean()).item()) <= 1e-12 * bnorm


def test_noalloc_residual_of_a_solve_is_the_reported_relres():
    g = gg.grid2d(64, weights="uniform", lo=1.0, hi=2.0, seed=1)
    h = P.lap_setup(g, seed=17)
    b = _dev(gg.rhs(g.n, seed=2))
    x = torch.empty_like(b)
    info = P.lap_pcg_solve(h, b, x)                       # existing entry point: the solve
    assert info.status == 0
    r = torch.empty_like(b)
    st, rnorm, bnorm = P.lap_laplacian_residual_noalloc(_dev(g.row_ptr, torch.int64),
                                                        _dev(g.col_idx, torch.int32), _dev(g.w),
                                                        x, b, r)
    assert st == 0
    assert abs(rnorm / bnorm - info.relres) <= 1e-3 * info.relres
    assert rnorm / bnorm <= 1e-8


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # rejected on the host before anything is queued (the pointers are never read)
    fake = 1 << 40
    norms = (P.C.c_double * 2)()
    st = P.lib().lap_laplacian_residual_noalloc((1 << 24) + 1, fake, fake, fake, fake, fake,
                                                fake, norms, None)
    assert st == 12                                       # LAP_ERR_UNSUPPORTED


def test_noalloc_calls_leave_device_memory_unchanged():
    """After a first call (which may load the library's device code), more
    calls change neither the device's free memory nor torch's allocator."""
    g = gg.grid2d(96, 80, weights="loguniform", lo=1e-2, hi=1e2, seed=4)
    rp = _dev(g.row_ptr, torch.int64)
    ci = _dev(g.col_idx, torch.int32)
    w = _dev(g.w)
    x = _dev(gg.rhs(g.n, seed=1))
    b = _dev(gg.rhs(g.n, seed=2))
    r = torch.empty_like(x)
    st, _, _ = P.lap_laplacian_residual_noalloc(rp, ci, w, x, b, r)
    assert st == 0
    r0 = r.clone()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    torch_bytes0 = torch.cuda.memory_allocated()
    for _ in range(3):
        st, _, _ = P.lap_laplacian_residual_noalloc(rp, ci, w, x, b, r)
        assert st == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == torch_bytes0
    assert torch.equal(r, r0)                         # deterministic partial sums
