"""The SELL-32 layout behind every matvec, checked on the host: the level-1
Laplacian and PEGP's L_H of grids, power-law, R-MAT, random geometric, star
and path graphs store every row's entries exactly once and in CSR order (in a
slice lane or, for long rows, in 128-entry-padded chunks), with weight-0
padding on the row itself (tests/sell_layout_check.cpp, compiled against
setup.cpp)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2207_07847_gb300", "csrc")

GRAPHS = [
    ("grid2d", lambda: gg.grid2d(64, weights="uniform", lo=1, hi=2, seed=1)),
    ("grid3d", lambda: gg.grid3d(20, weights="loguniform", lo=1e-3, hi=1e3, seed=3)),
    ("chunglu", lambda: gg.chung_lu(20000, avg_deg=16, seed=4)),
    ("rmat", lambda: gg.rmat(12, 16, seed=5)),
    ("rgg", lambda: gg.rgg(5000, seed=6)),
    ("star", lambda: gg.star(2000)),
    ("path", lambda: gg.path(3000)),
]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("sell") / "sell_layout_check")
    cmd = [cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           os.path.join(ROOT, "tests", "sell_layout_check.cpp"), os.path.join(CSRC, "setup.cpp"),
           "-o", out, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return out


@pytest.mark.parametrize("name,make", GRAPHS, ids=[g[0] for g in GRAPHS])
def test_sell_layout_stores_every_entry_once(checker, tmp_path, name, make):
    g = make()
    path = str(tmp_path / f"{name}.bin")
    with open(path, "wb") as f:
        np.array([g.n, len(g.col_idx)], dtype=np.int64).tofile(f)
        np.asarray(g.row_ptr, dtype=np.int64).tofile(f)
        np.asarray(g.col_idx, dtype=np.int32).tofile(f)
        np.asarray(g.w, dtype=np.float64).tofile(f)
    r = subprocess.run([checker, path], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith(("L1 ", "L_H "))]
    assert lines and lines[0].startswith("L1 ")
    if name in ("chunglu", "rmat", "star"):           # hub rows: the long-row chunks are exercised
        assert any(" long rows 0 " not in ln for ln in lines), r.stdout
