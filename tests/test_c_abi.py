"""The boundary as a C program sees it: include/lap.h compiles as C11 with all
warnings as errors, and a program linked against liblap.so sets up a graph
on the host (host_only, no GPU), reads the hierarchy and checks it against the
oracle's."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

P = pytest.importorskip("paper_2207_07847_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <stdlib.h>
#include "lap.h"

/* a 2D grid, 4-neighbour, weight 1 + ((i * 7 + j * 13) % 10) / 10 per edge */
int main(int argc, char **argv)
{
    if (argc < 3) return 9;
    const int nx = atoi(argv[1]), ny = atoi(argv[2]);
    const int64_t n = (int64_t)nx * ny;
    int64_t *rp = calloc((size_t)n + 1, sizeof *rp);
    int32_t *ci = malloc((size_t)n * 4 * sizeof *ci);
    double *w = malloc((size_t)n * 4 * sizeof *w);
    int64_t e = 0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const int64_t u = (int64_t)y * nx + x;
            const int64_t nb[4] = {y > 0 ? u - nx : -1, x > 0 ? u - 1 : -1,
                                   x + 1 < nx ? u + 1 : -1, y + 1 < ny ? u + nx : -1};
            for (int t = 0; t < 4; ++t) {
                if (nb[t] < 0) continue;
                const int64_t a = u < nb[t] ? u : nb[t], b = u < nb[t] ? nb[t] : u;
                ci[e] = (int32_t)nb[t];
                w[e++] = 1.0 + (double)((a * 7 + b * 13) % 10) / 10.0;
            }
            rp[u + 1] = e;
        }
    lap_options o;
    lap_options_default(&o);
    o.host_only = 1;
    o.seed = 3;
    lap_handle h = NULL;
    lap_status st = lap_setup(n, rp, ci, w, &o, NULL, &h);
    if (st != LAP_OK) {
        printf("setup %d %s\n", (int)st, lap_status_string(st));
        return 1;
    }
    lap_hierarchy_info info;
    if (lap_get_hierarchy_info(h, &info) != LAP_OK) return 2;
    printf("levels %d ntilde %lld\n", (int)info.levels, (long long)info.ntilde);
    int32_t *agg = malloc((size_t)n * sizeof *agg);
    int32_t *pa = malloc((size_t)n * sizeof *pa), *pb = malloc((size_t)n * sizeof *pb);
    if (lap_get_aggregates(h, 1, agg, pa, pb) != LAP_OK) return 3;
    for (int64_t u = 0; u < n; ++u) printf("%d\n", (int)agg[u]);
    /* errors come back as statuses */
    lap_handle bad = NULL;
    rp[1] = rp[1] + 1;
    printf("invalid %d\n", (int)lap_setup(n, rp, ci, w, &o, NULL, &bad));
    lap_destroy(h);
    free(rp); free(ci); free(w); free(agg); free(pa); free(pb);
    return 0;
}
"""


def test_header_compiles_as_c_and_host_setup_runs(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2207_07847_gb300 import build
    lib = build.build()
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I",
                    os.path.join(ROOT, "include"), str(src), lib, "-o", str(exe),
                    "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    nx, ny = 17, 11
    out = subprocess.run([str(exe), str(nx), str(ny)], capture_output=True, text=True,
                         check=True).stdout.split("\n")
    head = out[0].split()
    agg = np.array([int(v) for v in out[1:1 + nx * ny]])
    invalid = int(out[1 + nx * ny].split()[1])
    # the same graph through the oracle
    rp, ci, w = [0], [], []
    for y in range(ny):
        for x in range(nx):
            u = y * nx + x
            for v in (u - nx if y > 0 else -1, u - 1 if x > 0 else -1,
                      u + 1 if x + 1 < nx else -1, u + nx if y + 1 < ny else -1):
                if v < 0:
                    continue
                a, b = min(u, v), max(u, v)
                ci.append(v)
                w.append(1.0 + ((a * 7 + b * 13) % 10) / 10.0)
            rp.append(len(ci))
    ho = oracle.build_hierarchy(np.array(rp), np.array(ci), np.array(w), seed=3)
    assert int(head[1]) == ho.levels and int(head[3]) == ho.ntilde
    np.testing.assert_array_equal(agg, ho.agg[0])
    assert invalid != 0
