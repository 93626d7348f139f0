"""The library's host routines behind lap_estimate_condition, checked on the
CPU: the Lanczos tridiagonal built from CG's coefficients and its extreme
eigenvalues by Sturm-count bisection, against a dense eigensolve (numpy) of
the same matrices.  The routines are compiled from the library's source into
a small test driver."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2207_07847_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "lap_internal.h"
int main()
{
    int k, mode;
    while (std::scanf("%d %d", &mode, &k) == 2) {
        std::vector<double> a(k), b(k > 0 ? k - 1 : 0);
        if (mode == 0) {                       // tridiagonal given directly
            for (auto &x : a) std::scanf("%lf", &x);
            for (auto &x : b) std::scanf("%lf", &x);
        } else {                               // CG coefficients alpha, beta
            std::vector<double> al(k), be(k);
            for (auto &x : al) std::scanf("%lf", &x);
            for (auto &x : be) std::scanf("%lf", &x);
            if (!lap::lanczos_tridiagonal(al.data(), be.data(), k, a, b)) {
                std::printf("bad\n");
                continue;
            }
        }
        double lo = 0, hi = 0;
        if (!lap::tridiag_extremes(a, b, &lo, &hi)) std::printf("bad\n");
        else std::printf("%.17g %.17g\n", lo, hi);
    }
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("spectrum")
    src = d / "main.cpp"
    src.write_text(DRIVER)
    exe = d / "spectrum"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    str(src), os.path.join(CSRC, "spectrum.cpp"), "-o", str(exe)], check=True)

    def run(cases):
        lines = []
        for mode, k, xs in cases:
            lines.append(f"{mode} {k} " + " ".join(repr(float(x)) for x in xs))
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout.split("\n")
        return [None if ln.strip() == "bad" else tuple(map(float, ln.split()))
                for ln in out if ln.strip()]
    return run


def _dense(a, b):
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    ev = np.linalg.eigvalsh(T)
    return ev[0], ev[-1]


def test_bisection_matches_dense_eigensolve(driver):
    rng = np.random.default_rng(3)
    cases, want = [], []
    for k in (1, 2, 3, 7, 40, 300):
        a = rng.uniform(-2, 5, k)
        b = rng.uniform(-1, 1, k - 1) * (rng.uniform(0, 1, k - 1) > 0.1)   # some zero couplings
        cases.append((0, k, np.r_[a, b]))
        want.append(_dense(a, b))
    got = driver(cases)
    for (lo, hi), (wlo, whi) in zip(got, want):
        scale = max(abs(wlo), abs(whi))
        assert abs(lo - wlo) <= 1e-13 * scale and abs(hi - whi) <= 1e-13 * scale


def test_lanczos_tridiagonal_from_cg_coefficients(driver):
    """Plain CG on a path Laplacian (n = 30): the library's tridiagonal from
    alpha, beta has the path's extreme eigenvalues 2 - 2 cos(pi k / n) after
    n - 1 steps; inadmissible coefficients are refused."""
    n = 30
    L = np.diag(np.r_[1.0, 2.0 * np.ones(n - 2), 1.0]) - np.eye(n, k=1) - np.eye(n, k=-1)
    rng = np.random.default_rng(1)
    r = rng.standard_normal(n)
    r -= r.mean()
    x, p, rho = np.zeros(n), r.copy(), r @ r
    al, be = [], []
    for _ in range(n - 1):
        q = L @ p
        a = rho / (p @ q)
        r = r - a * q
        rn = r @ r
        al.append(a)
        be.append(rn / rho)
        p = r + be[-1] * p
        rho = rn
    k = len(al)
    got = driver([(1, k, np.r_[al, be]), (1, 2, [1.0, -1.0, 0.5, 0.0])])
    lo, hi = got[0]
    assert lo == pytest.approx(2 - 2 * np.cos(np.pi / n), rel=1e-8)
    assert hi == pytest.approx(2 - 2 * np.cos(np.pi * (n - 1) / n), rel=1e-10)
    assert got[1] is None
