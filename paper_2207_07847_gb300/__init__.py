"""Python binding of the GB300 graph-Laplacian solver library (``include/lap.h``).

Argument marshalling only: every step of setup and solve runs inside
``_lib/liblap.so`` (host C++ setup, CUDA kernels for sm_103a).  There is no
Python or CPU fallback: if the library has not been built, every entry point
raises ``LapLibraryMissing``.  Build it with ``paper_2207_07847_gb300.build``.

Device vectors are passed as CUDA tensors (float64, contiguous) or raw device
pointers (int); streams as ``torch.cuda.Stream`` or raw ``cudaStream_t`` ints.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblap.so")

LAP_PREC = {"none": 0, "msp": 1, "pegp_inner": 2, "pegp_exact": 3}
LAP_PRECISION = {"fp64": 0, "mixed": 1}
LAP_KRYLOV = {"cg": 0, "fgmres": 1}
LAP_MATCHING = {"greedy": 0, "handshake": 1}
STATUS = {0: "ok", 1: "invalid argument", 2: "not symmetric", 3: "not connected",
          4: "bad weight", 5: "out of memory", 6: "CUDA error", 7: "no convergence",
          8: "breakdown", 9: "timeout", 10: "cancelled", 11: "busy", 12: "unsupported"}
LAP_OK = 0


class LapLibraryMissing(RuntimeError):
    pass


class LapError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        super().__init__(f"{where}: lap status {status} ({STATUS.get(int(status), '?')})")


class lap_options(C.Structure):
    _fields_ = [("prec", C.c_int32), ("precision", C.c_int32), ("mu", C.c_double),
                ("coarse_max", C.c_int32), ("max_levels", C.c_int32), ("seed", C.c_uint64),
                ("order_random", C.c_int32), ("tol", C.c_double), ("maxit", C.c_int32),
                ("inner_tol", C.c_double), ("inner_maxit", C.c_int32),
                ("refine_tol", C.c_double), ("max_refine", C.c_int32),
                ("check_every", C.c_int32), ("timeout_s", C.c_double),
                ("spmv_tpr", C.c_int32), ("host_only", C.c_int32),
                ("stall_window", C.c_int32), ("krylov", C.c_int32), ("restart", C.c_int32),
                ("matching", C.c_int32), ("setup_device", C.c_int32), ("reserved", C.c_int32 * 1)]


class lap_solve_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("refinements", C.c_int32),
                ("inner_iterations", C.c_int32), ("restarts", C.c_int32),
                ("kernel_launches", C.c_int32), ("relres", C.c_double),
                ("relres_recurrence", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if not f.startswith("reserved")}


class lap_hierarchy_info(C.Structure):
    _fields_ = [("levels", C.c_int32), ("prec", C.c_int32), ("n", C.c_int64),
                ("ntilde", C.c_int64), ("nnz", C.c_int64), ("level_size", C.c_int64 * 64),
                ("nnz_H", C.c_int64), ("edges_T", C.c_int64), ("device_bytes", C.c_int64),
                ("mu", C.c_double)]


class lap_server_options(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_slots", C.c_int32),
                ("check_every", C.c_int32), ("reserved", C.c_int32 * 8)]


LAP_DONE_CB = C.CFUNCTYPE(None, C.c_void_p, C.c_uint64, C.POINTER(lap_solve_info))
_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

_lib = None

# (name, restype, argtypes) of every entry point declared in include/lap.h
_VP, _I32, _I64, _U64, _D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
SIGNATURES = [
    ("lap_options_default", None, [C.POINTER(lap_options)]),
    ("lap_status_string", C.c_char_p, [_I32]),
    ("lap_set_allocator", _I32, [_ALLOC_FN, _FREE_FN, _VP]),
    ("lap_setup", _I32, [_I64, _VP, _VP, _VP, C.POINTER(lap_options), _VP, C.POINTER(_VP)]),
    ("lap_destroy", None, [_VP]),
    ("lap_update_options", _I32, [_VP, C.POINTER(lap_options)]),
    ("lap_kernel_bench", _I32, [_VP, _I32, _I32, _I32, C.POINTER(_D), C.POINTER(_D)]),
    ("lap_get_hierarchy_info", _I32, [_VP, C.POINTER(lap_hierarchy_info)]),
    ("lap_get_aggregates", _I32, [_VP, _I32, _VP, _VP, _VP]),
    ("lap_get_expanded_edges", _I32, [_VP, _I32, _I64, C.POINTER(_I64), _VP, _VP, _VP]),
    ("lap_laplacian_apply", _I32, [_VP, _VP, _VP, _VP]),
    ("lap_precond_apply", _I32, [_VP, _VP, _VP, _VP]),
    ("lap_restrict_apply", _I32, [_VP, _VP, _VP, _VP]),
    ("lap_prolong_apply", _I32, [_VP, _VP, _VP, _VP]),
    ("lap_msp_solve", _I32, [_VP, _VP, _VP, _VP]),
    ("lap_pegp_apply", _I32, [_VP, _VP, _VP, _VP]),
    ("lap_pcg_solve", _I32, [_VP, _VP, _VP, _VP, C.POINTER(lap_solve_info)]),
    ("lap_get_history", _I32, [_VP, _VP, _I32, C.POINTER(_I32)]),
    ("lap_get_lanczos", _I32, [_VP, _VP, _VP, _I32, C.POINTER(_I32)]),
    ("lap_estimate_condition", _I32, [_VP, C.POINTER(_I32), C.POINTER(_D), C.POINTER(_D)]),
    ("lap_estimate_stretch", _I32, [_VP, _I32, _U64, _VP]),
    ("lap_pcg_solve_host", _I32, [_VP, _VP, _VP, _VP, C.POINTER(lap_solve_info)]),
    ("lap_pcg_solve_batched", _I32, [_I32, _VP, _VP, _VP, _VP, _VP, C.POINTER(lap_solve_info)]),
    ("lap_laplacian_residual_noalloc", _I32, [_I64, _VP, _VP, _VP, _VP, _VP, _VP,
                                               C.POINTER(_D), _VP]),
    ("lap_group_create", _I32, [_I32, _VP, C.POINTER(_VP)]),
    ("lap_pcg_solve_group", _I32, [_VP, _VP, _VP, _VP, _VP, C.POINTER(lap_solve_info)]),
    ("lap_group_destroy", None, [_VP]),
    ("lap_server_options_default", None, [C.POINTER(lap_server_options)]),
    ("lap_server_create", _I32, [C.POINTER(lap_server_options), C.POINTER(_VP)]),
    ("lap_serve_submit", _I32, [_VP, _VP, _I32, _VP, _VP, LAP_DONE_CB, _VP, C.POINTER(_U64)]),
    ("lap_serve_wait", _I32, [_VP, _U64, _D, C.POINTER(lap_solve_info)]),
    ("lap_serve_cancel", _I32, [_VP, _U64]),
    ("lap_server_destroy", None, [_VP]),
]


def lib():
    """Load the built library (raises LapLibraryMissing if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LapLibraryMissing(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -m paper_2207_07847_gb300.build)")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def build_library(force=False):
    """Compile liblap.so in-tree (nvcc, sm_103a)."""
    from . import build as _b
    return _b.build(force=force)


# ---------------------------------------------------------------------------
def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def make_options(**kw) -> lap_options:
    o = lap_options()
    lib().lap_options_default(C.byref(o))
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = LAP_PREC[v]
        if k == "precision" and isinstance(v, str):
            v = LAP_PRECISION[v]
        if k == "krylov" and isinstance(v, str):
            v = LAP_KRYLOV[v]
        if k == "matching" and isinstance(v, str):
            v = LAP_MATCHING[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


class Handle:
    """Owns a lap_handle; destroyed with the object or by close()."""

    def __init__(self, ptr, n, opts):
        self.ptr = ptr
        self.n = n
        self.opts = opts

    def close(self):
        if self.ptr:
            lib().lap_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return C.c_void_p(self.ptr)


def _check(status, where):
    if status != LAP_OK:
        raise LapError(status, where)


def lap_setup(row_ptr, col_idx=None, w=None, stream=None, **opts) -> Handle:
    """lap_setup on a host CSR graph: a graphgen.Graph, a scipy.sparse
    adjacency matrix (symmetric, positive off-diagonal weights, no diagonal),
    or the three CSR arrays."""
    if col_idx is None:
        g = row_ptr
        if hasattr(g, "tocsr"):                    # scipy.sparse
            g = g.tocsr()
            row_ptr, col_idx, w = g.indptr, g.indices, g.data
        else:
            row_ptr, col_idx, w = g.row_ptr, g.col_idx, g.w
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    o = make_options(**opts)
    out = C.c_void_p()
    st = lib().lap_setup(rp.shape[0] - 1, rp.ctypes.data, ci.ctypes.data, ww.ctypes.data,
                         C.byref(o), _stream(stream), C.byref(out))
    _check(st, "lap_setup")
    return Handle(out.value, rp.shape[0] - 1, o)


def lap_setup_status(row_ptr, col_idx, w, **opts) -> int:
    """lap_setup returning only the status (for validation tests)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    o = make_options(**opts)
    out = C.c_void_p()
    st = lib().lap_setup(rp.shape[0] - 1, rp.ctypes.data, ci.ctypes.data, ww.ctypes.data,
                         C.byref(o), None, C.byref(out))
    if st == LAP_OK:
        lib().lap_destroy(out)
    return st


def lap_destroy(h: Handle):
    h.close()


def lap_update_options(h: Handle, **opts):
    """Change solve-time options (see include/lap.h); returns the new options."""
    o = lap_options()
    C.memmove(C.byref(o), C.byref(h.opts), C.sizeof(lap_options))
    for k, v in opts.items():
        if k == "precision" and isinstance(v, str):
            v = LAP_PRECISION[v]
        if k == "krylov" and isinstance(v, str):
            v = LAP_KRYLOV[v]
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    _check(lib().lap_update_options(h, C.byref(o)), "lap_update_options")
    h.opts = o
    return o


KERNELS = {"spmv_L": 0, "spmv_LH": 1, "msp_sweep": 2, "update_up1": 3, "msp_tail": 4,
           "band_down1": 5, "pegp_gemv": 6, "inner_iteration": 7, "msp_tilde": 8,
           "spmv_LH_diag": 9}


def lap_kernel_bench(h: Handle, kernel, precision=0, reps=20):
    """(ms per launch, algorithmic bytes per launch) of one solver kernel."""
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    ms, by = C.c_double(), C.c_double()
    _check(lib().lap_kernel_bench(h, k, int(precision), int(reps), C.byref(ms), C.byref(by)),
           "lap_kernel_bench")
    return ms.value, by.value


def lap_get_hierarchy_info(h: Handle) -> dict:
    info = lap_hierarchy_info()
    _check(lib().lap_get_hierarchy_info(h, C.byref(info)), "lap_get_hierarchy_info")
    d = {f: getattr(info, f) for f, _ in info._fields_ if f != "level_size"}
    d["level_size"] = [int(info.level_size[k]) for k in range(info.levels)]
    return d


def lap_get_aggregates(h: Handle, level: int):
    """(agg, pair_a, pair_b) of level `level` (1-based, < levels)."""
    info = lap_get_hierarchy_info(h)
    nk, nk1 = info["level_size"][level - 1], info["level_size"][level]
    agg = np.empty(nk, dtype=np.int32)
    pa = np.empty(nk1, dtype=np.int32)
    pb = np.empty(nk1, dtype=np.int32)
    _check(lib().lap_get_aggregates(h, level, agg.ctypes.data, pa.ctypes.data, pb.ctypes.data),
           "lap_get_aggregates")
    return agg, pa, pb


def lap_get_expanded_edges(h: Handle, which: int):
    """Edges (i, j, w) with i < j of H (which=0) or T (which=1)."""
    cnt = C.c_int64()
    _check(lib().lap_get_expanded_edges(h, which, 0, C.byref(cnt), None, None, None), "count")
    i = np.empty(cnt.value, dtype=np.int64)
    j = np.empty(cnt.value, dtype=np.int64)
    w = np.empty(cnt.value, dtype=np.float64)
    _check(lib().lap_get_expanded_edges(h, which, cnt.value, C.byref(cnt), i.ctypes.data,
                                        j.ctypes.data, w.ctypes.data), "lap_get_expanded_edges")
    return i, j, w


def _block(name):
    def f(h: Handle, src, dst, stream=None):
        _check(getattr(lib(), name)(h, _ptr(src), _ptr(dst), _stream(stream)), name)
        return dst
    f.__name__ = name
    f.__doc__ = f"{name}(handle, src, dst, stream=None): see include/lap.h"
    return f


lap_laplacian_apply = _block("lap_laplacian_apply")
lap_precond_apply = _block("lap_precond_apply")
lap_restrict_apply = _block("lap_restrict_apply")
lap_prolong_apply = _block("lap_prolong_apply")
lap_msp_solve = _block("lap_msp_solve")
lap_pegp_apply = _block("lap_pegp_apply")


def lap_pcg_solve(h: Handle, b, x, stream=None) -> lap_solve_info:
    info = lap_solve_info()
    lib().lap_pcg_solve(h, _ptr(b), _ptr(x), _stream(stream), C.byref(info))
    return info


def lap_get_history(h: Handle):
    """Recurrence relative residuals of the last solve (numpy array)."""
    cnt = C.c_int32()
    _check(lib().lap_get_history(h, None, 0, C.byref(cnt)), "lap_get_history")
    out = np.empty(cnt.value, dtype=np.float64)
    _check(lib().lap_get_history(h, out.ctypes.data, cnt.value, C.byref(cnt)), "lap_get_history")
    return out[:cnt.value]


def lap_get_lanczos(h: Handle):
    """(alpha, beta) of the last solve's first CG run (numpy arrays)."""
    cnt = C.c_int32()
    _check(lib().lap_get_lanczos(h, None, None, 0, C.byref(cnt)), "lap_get_lanczos")
    a = np.empty(cnt.value, dtype=np.float64)
    b = np.empty(cnt.value, dtype=np.float64)
    _check(lib().lap_get_lanczos(h, a.ctypes.data, b.ctypes.data, cnt.value, C.byref(cnt)),
           "lap_get_lanczos")
    return a[:cnt.value], b[:cnt.value]


def lap_estimate_condition(h: Handle):
    """(steps, lambda_min, lambda_max) of B L from the last solve's CG run."""
    k, lo, hi = C.c_int32(), C.c_double(), C.c_double()
    _check(lib().lap_estimate_condition(h, C.byref(k), C.byref(lo), C.byref(hi)),
           "lap_estimate_condition")
    return k.value, lo.value, hi.value


def lap_estimate_stretch(h: Handle, samples=16, seed=0):
    """Hutchinson samples z^T L_T^+ L_H z (numpy array); their mean estimates
    tr(L_T^+ L_H), the stretch of H over T."""
    out = np.empty(int(samples), dtype=np.float64)
    _check(lib().lap_estimate_stretch(h, int(samples), int(seed), out.ctypes.data),
           "lap_estimate_stretch")
    return out


def lap_pcg_solve_host(h: Handle, b, x, stream=None) -> lap_solve_info:
    """Host vectors (numpy float64 or pinned CPU tensors); copies inside the call."""
    info = lap_solve_info()
    lib().lap_pcg_solve_host(h, _ptr(b), _ptr(x), _stream(stream), C.byref(info))
    return info


def lap_pcg_solve_batched(handles, Bs, Xs, stream=None):
    """Batched solve: handles[g] with Bs[g] (n_g x nrhs_g column-major, i.e. a
    (nrhs_g, n_g) row-major tensor) and outputs Xs[g] of the same shape."""
    ng = len(handles)
    hs = (C.c_void_p * ng)(*[h.ptr for h in handles])
    nr = (C.c_int32 * ng)(*[int(B.shape[0]) if B.dim() == 2 else 1 for B in Bs])
    pb = (C.c_void_p * ng)(*[_ptr(B) for B in Bs])
    px = (C.c_void_p * ng)(*[_ptr(X) for X in Xs])
    tot = sum(nr)
    infos = (lap_solve_info * tot)()
    st = lib().lap_pcg_solve_batched(ng, hs, nr, pb, px, _stream(stream), infos)
    return st, list(infos)


class Group:
    """A solve group (lap_group_create): the handles' graphs merged for
    solves with one launch per PCG phase for all of them.  Keeps the handles
    alive as long as the group."""

    def __init__(self, handles):
        self.handles = list(handles)
        ng = len(self.handles)
        hs = (C.c_void_p * ng)(*[h.ptr for h in self.handles])
        p = C.c_void_p()
        _check(lib().lap_group_create(ng, hs, C.byref(p)), "lap_group_create")
        self.ptr = p.value

    def close(self):
        if getattr(self, "ptr", None):
            lib().lap_group_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lap_pcg_solve_group(group, Bs, Xs, stream=None):
    """Group solve: graph g's right-hand sides Bs[g] ((nrhs_g, n_g) row-major
    = n_g x nrhs_g column-major) into Xs[g]; (status, infos)."""
    ng = len(group.handles)
    nr = (C.c_int32 * ng)(*[int(B.shape[0]) if B.dim() == 2 else 1 for B in Bs])
    pb = (C.c_void_p * ng)(*[_ptr(B) for B in Bs])
    px = (C.c_void_p * ng)(*[_ptr(X) for X in Xs])
    infos = (lap_solve_info * max(sum(nr), 1))()
    st = lib().lap_pcg_solve_group(group.ptr, nr, pb, px, _stream(stream), infos)
    return st, list(infos)[:sum(nr)]


def lap_laplacian_residual_noalloc(row_ptr, col_idx, w, x, b, r, stream=None):
    """r = Pi b - L x on device CSR / vectors with no device allocation;
    returns (status, ||r||, ||Pi b||).  See include/lap.h."""
    norms = (C.c_double * 2)()
    n = int(row_ptr.shape[0]) - 1
    st = lib().lap_laplacian_residual_noalloc(n, _ptr(row_ptr), _ptr(col_idx), _ptr(w), _ptr(x),
                                              _ptr(b), _ptr(r), norms, _stream(stream))
    return st, norms[0], norms[1]


# ---------------------------------------------------------------------------
_torch_alloc_refs = None


def set_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _torch_alloc_refs
    import torch

    def _alloc(ctx, nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device())
        except Exception:
            return None

    def _free(ctx, ptr, stream):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass

    a, f = _ALLOC_FN(_alloc), _FREE_FN(_free)
    _check(lib().lap_set_allocator(a, f, None), "lap_set_allocator")
    _torch_alloc_refs = (a, f)


def clear_allocator():
    global _torch_alloc_refs
    _check(lib().lap_set_allocator(_ALLOC_FN(), _FREE_FN(), None), "lap_set_allocator")
    _torch_alloc_refs = None


def lap_server_options_default() -> lap_server_options:
    o = lap_server_options()
    lib().lap_server_options_default(C.byref(o))
    return o


class Server:
    """A continuous-batching solve server (lap_server_*).

    ``submit(h, B, X)`` queues L_h X = B for a (nrhs, n) float64 CUDA tensor B
    (one right-hand side per row, i.e. the column-major layout of the C ABI)
    and returns the request id; ``wait(id)`` blocks until it finished and
    returns ``(status, info)``.  The tensors and the optional callback are kept
    alive here until the request has been waited for or the server closed.
    """

    def __init__(self, hbm_budget_bytes=None, max_slots=None, check_every=None):
        o = lap_server_options_default()
        if hbm_budget_bytes is not None:
            o.hbm_budget_bytes = int(hbm_budget_bytes)
        if max_slots is not None:
            o.max_slots = int(max_slots)
        if check_every is not None:
            o.check_every = int(check_every)
        self.options = o
        p = C.c_void_p()
        _check(lib().lap_server_create(C.byref(o), C.byref(p)), "lap_server_create")
        self.ptr = p.value
        self._keep = {}

    def submit(self, h: Handle, B, X, callback=None) -> int:
        nrhs = int(B.shape[0]) if B.dim() == 2 else 1
        cb = LAP_DONE_CB(lambda user, rid, info: callback(int(rid), info.contents.as_dict())) \
            if callback is not None else LAP_DONE_CB()
        rid = C.c_uint64(0)
        st = lib().lap_serve_submit(self.ptr, h.ptr, nrhs, _ptr(B), _ptr(X), cb, None, C.byref(rid))
        _check(st, "lap_serve_submit")
        self._keep[rid.value] = (B, X, cb)
        return rid.value

    def wait(self, rid: int, timeout_s: float = 0.0):
        info = lap_solve_info()
        info.status = -1                  # stays -1 while the request runs
        st = lib().lap_serve_wait(self.ptr, rid, float(timeout_s), C.byref(info))
        if info.status != -1 or st == 1:  # finished (or unknown id)
            self._keep.pop(rid, None)
        return st, info

    def cancel(self, rid: int) -> int:
        return lib().lap_serve_cancel(self.ptr, rid)

    def close(self):
        if self.ptr:
            lib().lap_server_destroy(self.ptr)
            self.ptr = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
