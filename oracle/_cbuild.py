"""ORACLE -- test infrastructure only.  Builds and loads the oracle's plain C
part (``hier.c``) with the host C compiler; no CUDA, no shared code with the
solver library."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hier.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_OUT = os.path.join(_OUT_DIR, "liboracle_hier.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile hier.c into a shared object (idempotent)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        cc = os.environ.get("CC", "gcc")
        subprocess.check_call([cc, "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            i64, i32, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
            vp = ctypes.c_void_p
            L.oh_splitmix64.restype = u64
            L.oh_splitmix64.argtypes = [u64, u64]
            L.oh_visit_order.restype = None
            L.oh_visit_order.argtypes = [i64, u64, i32, i32, vp]
            L.oh_match.restype = i64
            L.oh_match.argtypes = [i64, vp, vp, vp, u64, i32, i32, vp, vp, vp]
            L.oh_coarse.restype = i64
            L.oh_coarse.argtypes = [i64, vp, vp, vp, vp, i64, vp, vp, vp]
            _lib = L
    return _lib
