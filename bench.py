#!/usr/bin/env python
"""Benchmark: preconditioned CG solves per second at relative residual 1e-8.

Workload (one "step" = one full solve of L x = b, setup excluded): the 3D
128^3 7-point grid graph (2,097,152 vertices, 6,242,304 edges) with edge
weights log-uniform in [1e-3, 1e3], one N(0,1) right-hand side per step
(projected to mean zero by the solver), PCG preconditioned by the paper's
PEGP (inner CG on L_H with the MSP sparsifier, mu = 0.8), mixed precision:
FP32 matvecs/sweeps with FP32 accumulation, FP64 dots, scalars, projection,
coarsest solve and iterative-refinement residuals.  The plain FP64 solve of
the same system is measured beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own copy ("replicas only"; no
collective on the data path) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PCG solves/s at relres 1e-8 and HBM GB/s vs peak; p50/p99 latency vs plain FP64"
WORKLOAD = {
    "name": "grid3d_128^3_loguniform[1e-3,1e3]_PEGP_mu0.8",
    "nx": 128, "wlo": 1e-3, "whi": 1e3, "wseed": 3, "prec": "pegp_inner", "mu": 0.8,
    "tol": 1e-8, "inner_tol": 1e-1, "inner_maxit": 12, "setup_seed": 1,
}
FP64_ALU_PEAK_TFLOPS = 1.25     # nominal FP64 rate of a GB300 (no measured figure exists)
# DRAM bytes per launch of the dominant kernel from an ncu capture of the current
# kernel, scaled to the 128^3 workload (profiles/k_sell_f32_LH_grid3d96.md);
# removed whenever the kernel changes.
MEASURED_TRAFFIC = {"spmv_LH": 1.803e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--aux-steps", type=int, default=5,
                    help="timed solves of the FP64 comparison, e2e and MSP lines")
    ap.add_argument("--profile", type=int, default=0,
                    help="profiling run: one solve of each kind capped at this many outer "
                         "iterations, nothing timed or printed")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=WORKLOAD["nx"], help="grid side (128 = the workload)")
    ap.add_argument("--prec", default=WORKLOAD["prec"],
                    choices=["pegp_inner", "msp", "none", "pegp_exact"],
                    help="pegp_exact: profiling runs only (small grids)")
    ap.add_argument("--exact-side", type=int, default=64,
                    help="side of the 2D grid of the exact-PEGP line (0: skip it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--powerlaw-n", type=int, default=1 << 20,
                    help="vertices of the Chung-Lu line (0: skip it)")
    ap.add_argument("--batched-scale", type=int, default=20,
                    help="R-MAT scale of the batched line (0: skip it)")
    ap.add_argument("--batched-rhs", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="requests of the serving line (0: skip it)")
    ap.add_argument("--serve-graphs", type=int, default=32)
    ap.add_argument("--serve-nmax", type=float, default=1e6)
    ap.add_argument("--serve-plain-s", type=float, default=60.0,
                    help="time limit of the plain FP64 comparison stream")
    ap.add_argument("--serve-load", type=float, default=0.7,
                    help="Poisson arrival rate as a fraction of the server's capacity measured by a "
                         "closed burst of the first 256 requests")
    ap.add_argument("--serving-only", action="store_true",
                    help="only the serving line (e.g. 10,000 requests over 64 graphs), printed alone")
    ap.add_argument("--only", default=None,
                    choices=["serving", "powerlaw", "batched", "group", "handshake", "pegp_exact"],
                    help="run this one auxiliary line alone and print it")
    ap.add_argument("--handshake", type=int, default=1,
                    help="1: also solve the headline grid with the deterministic parallel "
                         "matching variant (a method change; reported apart, 0: skip)")
    ap.add_argument("--group-graphs", type=int, default=16,
                    help="graphs of the solve-group line (0: skip)")
    ap.add_argument("--oracle-cap-s", type=float, default=40.0,
                    help="seconds of timed oracle iterations per oracle leg")
    ap.add_argument("--sweep-inner", action="store_true",
                    help="only sweep the PEGP inner cap and tolerance at the workload")
    ap.add_argument("--profile-batched", type=int, default=0,
                    help="profiling: one batched solve of the R-MAT workload (--batched-scale, "
                         "--batched-rhs) capped at this many iterations, inside the NVTX range 'batched'")
    ap.add_argument("--kernel-only", default=None,
                    help="profiling: set up the workload at --nx and time one lap_kernel_bench kernel "
                         "(FP32, one warm-up and --steps launches) inside the NVTX range 'kernel'")
    ap.add_argument("--oracle-worker", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
def ranks_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value, world, device=None):
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms_max):
    """Units per second of the whole job: every rank processed units_per_rank
    (replicas), the job took the slowest rank's ms_max."""
    return units_per_rank * world / (ms_max * 1e-3)


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [ln.strip().split(", ") for ln in self.file.read().splitlines() if ln.strip()]
        os.unlink(self.file.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
REF_OUTER_ITERATIONS = 2000   # outer iterations per solve assumed by the reference arm (see DESIGN)


def host_description():
    """CPU model and logical core count of this host."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "processor\t")) and ":" in ln:
                    v = ln.split(":", 1)[1].strip()
                    if ln.lower().startswith("model name") and v:
                        model = v
                        break
    except OSError:
        pass
    try:
        import subprocess as sp_
        out = sp_.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count(), "machine": platform.machine()}


def oracle_worker(spec_json):
    """Runs in its own process.  mode "capped": build the oracle preconditioner
    of the full workload (setup, not timed), report ready, optionally wait
    for a line on stdin, then run the oracle PCG for cap_s seconds and report
    the outer iterations completed (and their inner iterations).  mode
    "samples": oracle solutions of the reduced error-check systems, saved to
    spec["out"]."""
    spec = json.loads(spec_json)
    import numpy as np

    import graphgen as gg
    import oracle
    if spec["mode"] == "samples":
        sols = {}
        for name, (kind, g, mu, kw, seeds) in error_samples().items():
            for s_ in seeds:
                b = gg.rhs(g.n, seed=s_)
                res = oracle.solve(g, b, kind, mu=mu, seed=WORKLOAD["setup_seed"], maxit=20000, **kw)
                sols[f"{name}:{s_}"] = res.x
        np.savez(spec["out"], **sols)
        print(json.dumps({"done": len(sols)}), flush=True)
        return
    nx = spec["nx"]
    g = gg.grid3d(nx, weights="loguniform", lo=WORKLOAD["wlo"], hi=WORKLOAD["whi"], seed=WORKLOAD["wseed"])
    t0 = time.perf_counter()
    ho = oracle.build_hierarchy(g.row_ptr, g.col_idx, g.w, seed=WORKLOAD["setup_seed"])
    ops = oracle.expanded_operators(ho, WORKLOAD["mu"], with_LG=False)
    M = oracle.OraclePreconditioner(spec["prec"], ops, inner_tol=WORKLOAD["inner_tol"],
                                    inner_maxit=WORKLOAD["inner_maxit"])
    L = ops.L
    setup_s = time.perf_counter() - t0
    print(json.dumps({"ready": True, "setup_s": setup_s, "n": g.n}), flush=True)
    if spec.get("wait"):
        sys.stdin.readline()
    b = gg.rhs(g.n, seed=100)
    t0 = time.perf_counter()
    res = oracle.pcg(L, b, M, tol=WORKLOAD["tol"], maxit=10 ** 6, flexible=M.flexible,
                     deadline=t0 + spec["cap_s"])
    t = time.perf_counter() - t0
    print(json.dumps({"n": g.n, "outer": res.iters, "inner": int(sum(M.inner_iters)), "seconds": t,
                      "relres": res.history[-1] if res.history else 1.0, "setup_s": setup_s}), flush=True)


_WORKERS = []


def _kill_workers():
    for p_ in _WORKERS:
        if p_.poll() is None:
            p_.kill()


def start_oracle(nx, prec, cap_s, threads, wait):
    """A capped oracle worker in its own process (setup starts at once)."""
    th = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=th, OPENBLAS_NUM_THREADS=th, MKL_NUM_THREADS=th)
    spec = json.dumps({"mode": "capped", "nx": nx, "prec": prec, "cap_s": cap_s, "wait": wait})
    if not _WORKERS:
        import atexit
        atexit.register(_kill_workers)
    p_ = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-worker", spec],
                          stdin=subprocess.PIPE, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                          text=True, env=env)
    _WORKERS.append(p_)
    return p_


def finish_oracle(proc, timeout=1800):
    """Wait for the worker's setup, start its timed iterations, return its report."""
    ready = json.loads(proc.stdout.readline() or "{}")
    if not ready.get("ready"):
        proc.kill()
        raise RuntimeError("oracle worker failed: " + proc.stderr.read()[-1500:])
    proc.stdin.write("go\n")
    proc.stdin.flush()
    out, err = proc.communicate(timeout=timeout)
    if proc.returncode != 0:
        raise RuntimeError(err[-1500:])
    return json.loads(out.strip().splitlines()[-1])


def oracle_rate(rep, outer_per_solve):
    """Solves/s of the oracle from its timed outer iterations at the full
    workload and the outer iterations one solve takes."""
    per_iter = rep["seconds"] / max(rep["outer"], 1)
    return 1.0 / (per_iter * outer_per_solve), per_iter


def cpu_baseline(procs, n_full, outer_per_solve, source):
    """The oracle at the full workload, timed for a bounded number of outer
    iterations, single-threaded and with every core for its BLAS."""
    legs = {}
    for threads, proc in procs:
        rep = finish_oracle(proc)
        rate, per_iter = oracle_rate(rep, outer_per_solve)
        legs[threads] = (rate, per_iter, rep)
    best = max(legs, key=lambda t: legs[t][0])
    rate, per_iter, rep = legs[best]
    hd = host_description()
    desc = "; ".join(f"{t} thread(s): {l[2]['outer']} outer ({l[2]['inner']} inner) iterations in "
                     f"{l[2]['seconds']:.1f} s, {l[1]:.2f} s per outer iteration, {l[0]:.3g} solves/s"
                     for t, l in sorted(legs.items()))
    return {"value": rate, "unit": "solves/s", "cores": best, "kind": "oracle",
            "sample": (f"oracle (numpy/scipy PCG with the PEGP inner solve) on the full {n_full}-vertex "
                       f"workload, setup excluded ({rep['setup_s']:.0f} s), timed for a bounded number "
                       f"of outer iterations: {desc}; solves/s = 1 / (seconds per outer iteration x "
                       f"{outer_per_solve} outer iterations per solve, {source})"),
            "host": hd, "legs": {str(t): {"solves_per_s": l[0], "s_per_outer": l[1],
                                          "outer": l[2]["outer"], "seconds": l[2]["seconds"]}
                                 for t, l in legs.items()}}


def error_samples():
    """Reduced systems of each workload for the error against the FP64 oracle:
    name -> (preconditioner, graph, mu, options, right-hand side seeds)."""
    import graphgen as gg
    return {
        "grid2d_64_pegp_exact_fp64": ("pegp_exact", gg.grid2d(64, weights="uniform", lo=1.0, hi=2.0, seed=1),
                                      1 / 64, {}, (900, 901)),
        "grid3d_16_loguniform_pegp_inner_mixed": (
            "pegp_inner", gg.grid3d(16, weights="loguniform", lo=1e-3, hi=1e3, seed=3), 0.8,
            {"inner_tol": 0.1, "inner_maxit": 12}, (902,)),
        "chunglu_16384_msp_mixed": ("msp", gg.chung_lu(1 << 14, avg_deg=16.0, gamma=2.5, weights="uniform01",
                                                       seed=4), 0.8, {}, (903, 904)),
        "rmat_s12_msp_mixed_batched": ("msp", gg.rmat(12, 16, seed=5), 0.8, {}, (905, 906, 907, 908)),
    }


def start_samples(path):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    spec = json.dumps({"mode": "samples", "out": path})
    p_ = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-worker", spec],
                          stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
    _WORKERS.append(p_)
    return p_


def errors_vs_oracle(proc, path, dev):
    """||x_gpu - x_oracle|| / ||x_oracle|| on the reduced systems (GPU solves
    through the C ABI; the oracle's FP64 solutions from the sample worker)."""
    import numpy as np
    import torch

    import graphgen as gg
    import paper_2207_07847_gb300 as P
    out, err = proc.communicate(timeout=1800)
    if proc.returncode != 0:
        raise RuntimeError(err[-1500:])
    ref = np.load(path)
    res = {}
    for name, (kind, g, mu, kw, seeds) in error_samples().items():
        precision = "fp64" if name.endswith("fp64") else "mixed"
        opts = {k: v for k, v in kw.items()}
        h = P.lap_setup(g, prec=kind, mu=mu, precision=precision, seed=WORKLOAD["setup_seed"], maxit=20000,
                        **opts)
        B = torch.stack([torch.as_tensor(gg.rhs(g.n, seed=s_), device=dev) for s_ in seeds])
        X = torch.empty_like(B)
        if name.endswith("batched"):
            st, infos = P.lap_pcg_solve_batched([h], [B], [X])
        else:
            infos = [P.lap_pcg_solve(h, B[j], X[j]) for j in range(len(seeds))]
        torch.cuda.synchronize()
        errs = []
        for j, s_ in enumerate(seeds):
            xo = ref[f"{name}:{s_}"]
            errs.append(float(np.linalg.norm(X[j].cpu().numpy() - xo) / np.linalg.norm(xo)))
        res[name] = {"n": g.n, "columns": len(seeds), "error_max": max(errs),
                     "relres_max": max(i.relres for i in infos),
                     "status": [i.status for i in infos]}
        h.close()
    return res


# ---------------------------------------------------------------------------
def bench_ours(args, rank, world):
    import numpy as np
    import torch

    import graphgen as gg
    import paper_2207_07847_gb300 as P

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    if rank == 0:
        P.build_library()
    if world > 1:
        torch.distributed.barrier()
    P.lib()
    P.set_torch_allocator()
    if args.prec == "pegp_exact" and not args.profile:
        raise SystemExit("--prec pegp_exact is for profiling runs (--profile); the exact PEGP "
                         "is timed on the small 2D grid line (--exact-side)")

    # the oracle legs: their setups run on other host cores while the GPU is measured
    oracle_procs, samples = [], None
    if (rank == 0 and world == 1 and not args.no_cpu_baseline and not args.profile and not args.sweep_inner
            and not args.kernel_only and not args.profile_batched):
        try:
            oracle_procs = [(t, start_oracle(args.nx, args.prec, args.oracle_cap_s, t, True))
                            for t in (1, os.cpu_count() or 1)]
            path = os.path.join(tempfile.mkdtemp(), "oracle_samples.npz")
            samples = (start_samples(path), path)
        except Exception as e:
            print(f"[bench] oracle legs not started: {e}", file=sys.stderr)
    g = gg.grid3d(args.nx, weights="loguniform", lo=WORKLOAD["wlo"], hi=WORKLOAD["whi"],
                  seed=WORKLOAD["wseed"])
    if args.profile_batched:
        gb = gg.rmat(args.batched_scale, 16, seed=5)
        hb = P.lap_setup(gb, prec="msp", mu=WORKLOAD["mu"], precision="mixed", seed=WORKLOAD["setup_seed"],
                         tol=WORKLOAD["tol"], maxit=args.profile_batched)
        gen = torch.Generator(device=dev)
        gen.manual_seed(500)
        B = torch.randn(args.batched_rhs, gb.n, dtype=torch.float64, device=dev, generator=gen)
        X = torch.empty_like(B)
        P.lap_pcg_solve_batched([hb], [B], [X])                 # warm-up (autotune, graphs)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("batched")
        P.lap_pcg_solve_batched([hb], [B], [X])
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        hb.close()
        return None
    if args.sweep_inner:
        return sweep_inner(args, g, dev)
    if args.kernel_only:
        hk = P.lap_setup(g, prec=args.prec, mu=WORKLOAD["mu"], precision="mixed", seed=WORKLOAD["setup_seed"],
                         tol=WORKLOAD["tol"], inner_tol=WORKLOAD["inner_tol"],
                         inner_maxit=WORKLOAD["inner_maxit"])
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("kernel")
        ms, by = P.lap_kernel_bench(hk, args.kernel_only, 1, args.steps)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        hk.close()
        print(f"[bench] {args.kernel_only} at {args.nx}^3: {ms * 1e3:.1f} us, {by / 1e9:.4f} GB", file=sys.stderr)
        return None
    t0 = time.perf_counter()
    h = P.lap_setup(g, prec=args.prec, mu=WORKLOAD["mu"], precision="mixed",
                    seed=WORKLOAD["setup_seed"], tol=WORKLOAD["tol"],
                    inner_tol=WORKLOAD["inner_tol"], inner_maxit=WORKLOAD["inner_maxit"],
                    maxit=30000)
    setup_s = time.perf_counter() - t0
    if args.profile:
        # profiling: the kernel mix of each solve kind, few iterations, nothing timed
        b0 = torch.as_tensor(gg.rhs(g.n, seed=100), device=dev)
        x0 = torch.empty_like(b0)
        for precision in ("mixed", "fp64"):
            P.lap_update_options(h, precision=precision, maxit=args.profile)
            P.lap_pcg_solve(h, b0, x0)
        torch.cuda.synchronize()
        h.close()
        return None
    info_h = P.lap_get_hierarchy_info(h)
    K, W = args.steps, args.warmup
    rhs = [gg.rhs(g.n, seed=100 + i + 1000 * rank) for i in range(K + W + max(args.aux_steps, 1))]
    dB = [torch.as_tensor(b, device=dev) for b in rhs]
    hB = [torch.as_tensor(b).pin_memory() for b in rhs]
    x = torch.empty(g.n, dtype=torch.float64, device=dev)
    xh = torch.empty(g.n, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()

    def timed(precision, host=False, hh=None, k_steps=None, w_steps=None):
        hh = hh or h
        KK = K if k_steps is None else k_steps
        WW = W if w_steps is None else w_steps
        P.lap_update_options(hh, precision=precision)
        for i in range(WW):
            inf = (P.lap_pcg_solve_host(hh, hB[i], xh) if host else P.lap_pcg_solve(hh, dB[i], x))
            print(f"[bench] warmup {precision} host={host}: {inf.as_dict()}", file=sys.stderr,
                  flush=True)
        ranks_barrier(world)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos, lat = [], []
        ev0.record(stream)
        for i in range(W, W + KK):
            e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            inf = (P.lap_pcg_solve_host(hh, hB[i], xh) if host else P.lap_pcg_solve(hh, dB[i], x))
            e_b.record(stream)
            print(f"[bench] step {precision} host={host}: {inf.as_dict()}", file=sys.stderr,
                  flush=True)
            infos.append(inf)
            lat.append((e_a, e_b))
        ev1.record(stream)
        torch.cuda.synchronize()
        ranks_barrier(world)
        ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
        lats = sorted(a.elapsed_time(b) for a, b in lat)
        return ms, infos, lats

    def pct(v, q):
        return v[min(len(v) - 1, int(math.ceil(q * len(v))) - 1)]

    A = args.aux_steps
    clocks = ClockSampler(dev.index)
    clocks.start()
    ms_mixed, inf_mixed, lat_mixed = timed("mixed")
    clk = clocks.stop()
    ms_fp64, inf_fp64, lat_fp64 = timed("fp64", k_steps=A, w_steps=0)
    ms_e2e, inf_e2e, _ = timed("mixed", host=True, k_steps=A, w_steps=0)

    # dominant kernel: the FP32 L_H matvec of the inner solves (PEGP) or the FP32
    # L matvec (MSP / none); timed back to back on the solve's data with CUDA
    # events on the library's stream
    P.lap_update_options(h, precision="mixed")
    kern = "spmv_LH" if args.prec == "pegp_inner" else "spmv_L"
    kms, kbytes = P.lap_kernel_bench(h, kern, 1, 20)
    peak, peak_kind = measured_peaks()
    achieved = kbytes / (kms * 1e-3) / 1e9
    other = {}
    for name, prec in (("spmv_L_f32", ("spmv_L", 1)), ("spmv_L_f64", ("spmv_L", 0)),
                       ("msp_sweep_f32", ("msp_sweep", 1)), ("update_up1_f32", ("update_up1", 1))):
        m_, b_ = P.lap_kernel_bench(h, prec[0], prec[1], 20)
        other[name] = {"us": round(m_ * 1e3, 2), "GB/s": round(b_ / (m_ * 1e-3) / 1e9, 1)}
    if args.prec == "pegp_inner":
        m_, b_ = P.lap_kernel_bench(h, "spmv_LH", 0, 10)
        other["spmv_LH_f64"] = {"us": round(m_ * 1e3, 2), "GB/s": round(b_ / (m_ * 1e-3) / 1e9, 1)}
        # the stored-diagonal form of the same matvec (timed only; the solves
        # use the edge-difference form): one multiply-add per entry in place of
        # a subtraction and a multiply-add, one more vector read
        for pname, pid in (("f64", 0), ("f32", 1)):
            m_, b_ = P.lap_kernel_bench(h, "spmv_LH_diag", pid, 10)
            other[f"spmv_LH_diag_{pname}"] = {"us": round(m_ * 1e3, 2), "GB/s": round(b_ / (m_ * 1e-3) / 1e9, 1)}

    failed = [i.as_dict() for i in inf_mixed + inf_fp64 + inf_e2e if i.status != 0]
    # the paper's sparsifier alone (MSP) on the same system, for comparison
    msp = None
    if args.prec == "pegp_inner":
        hm = P.lap_setup(g, prec="msp", mu=WORKLOAD["mu"], precision="mixed",
                         seed=WORKLOAD["setup_seed"], tol=WORKLOAD["tol"], maxit=30000)
        ms_mm, inf_mm, lat_mm = timed("mixed", hh=hm, k_steps=A, w_steps=1)
        ms_mf, inf_mf, lat_mf = timed("fp64", hh=hm, k_steps=A, w_steps=0)
        # Lanczos estimate of B L's extreme eigenvalues from the last FP64 solve
        k_l, lo_l, hi_l = P.lap_estimate_condition(hm)
        msp = {"mixed": {"value": whole_job_rate(A, world, ms_mm), "unit": "solves/s",
                         "latency_ms": {"p50": pct(lat_mm, 0.5), "p99": pct(lat_mm, 0.99)},
                         "iterations": statistics.median(i.iterations for i in inf_mm)},
               "fp64": {"value": whole_job_rate(A, world, ms_mf), "unit": "solves/s",
                        "latency_ms": {"p50": pct(lat_mf, 0.5), "p99": pct(lat_mf, 0.99)},
                        "iterations": statistics.median(i.iterations for i in inf_mf),
                        "lanczos": {"steps": k_l, "lambda_min": lo_l, "lambda_max": hi_l,
                                    "kappa": hi_l / lo_l}},
               "failed": [i.as_dict() for i in inf_mm + inf_mf if i.status != 0]}
        hm.close()
    value = whole_job_rate(K, world, ms_mixed)
    fp64_value = whole_job_rate(A, world, ms_fp64)
    e2e_value = whole_job_rate(A, world, ms_e2e)
    it_mixed = statistics.median(i.iterations for i in inf_mixed)
    it_fp64 = statistics.median(i.iterations for i in inf_fp64)
    inner_fp64 = statistics.median(i.inner_iterations for i in inf_fp64)
    result = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms_mixed / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"] if args.nx == 128 else f"grid3d_{args.nx}^3",
                   "n": g.n, "nnz": info_h["nnz"], "levels": info_h["levels"],
                   "ntilde": info_h["ntilde"], "nnz_H": info_h["nnz_H"],
                   "preconditioner": args.prec, "mu": WORKLOAD["mu"], "tol": WORKLOAD["tol"],
                   "inner_tol": WORKLOAD["inner_tol"], "precision": "mixed (FP32 matvec/sweeps, "
                   "FP64 dots/scalars/refinement residuals)", "rhs": "N(0,1), one per step",
                   "l2": "inputs larger than L2 (L_H alone is "
                   f"{info_h['nnz_H'] * 8 / 1e9:.1f} GB in FP32)", "parallelism": f"replicas x{world}",
                   "setup_s": round(setup_s, 2)},
        "latency_ms": {"p50": pct(lat_mixed, 0.5), "p99": pct(lat_mixed, 0.99)},
        "iterations": {"outer": it_mixed, "refinements": statistics.median(i.refinements for i in inf_mixed),
                       "inner": statistics.median(i.inner_iterations for i in inf_mixed),
                       "relres_max": max(i.relres for i in inf_mixed)},
        "fp64": {"value": fp64_value, "unit": "solves/s", "latency_ms": {
            "p50": pct(lat_fp64, 0.5), "p99": pct(lat_fp64, 0.99)}, "iterations": it_fp64,
            "inner_iterations": inner_fp64, "relres_max": max(i.relres for i in inf_fp64)},
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": g.n * 8,
                "d2h_bytes_per_step": g.n * 8},
        "gpu_launches": int(sum(i.kernel_launches for i in inf_mixed)),
        "roofline": {"bound": "hbm", "kernel": f"{kern} (FP32)", "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_kind": peak_kind, "bytes_per_launch": kbytes,
                     "us_per_launch": round(kms * 1e3, 2),
                     "traffic": MEASURED_TRAFFIC.get(kern) if args.nx == 128 else None},
        "kernels": other,
        "clocks": clk,
        "msp_same_system": msp,
        "failed_solves": failed,
    }
    h.close()
    if args.exact_side > 0:
        result["pegp_exact"] = bench_pegp_exact(args, dev, world)
    if args.powerlaw_n > 0:
        result["powerlaw"] = bench_powerlaw(args, dev, world)
    if args.batched_scale > 0:
        result["batched"] = bench_batched(args, dev, world)
    if args.group_graphs > 0:
        result["group"] = bench_group(args, dev, world)
    if args.serve_requests > 0:
        result["serving"] = bench_serving(args, dev, world)
    if args.handshake:
        try:
            result["handshake_matching"] = bench_handshake(args, dev, world)
        except Exception as e:          # a variant line, never fatal to the report
            result["handshake_matching"] = {"error": str(e)[-300:]}
    if oracle_procs:
        try:
            result["cpu_baseline"] = cpu_baseline(
                oracle_procs, g.n, it_fp64,
                f"the median outer iterations of this run's FP64 arm on the GPU, the same iteration")
        except Exception as e:          # the baseline is reported, never fatal
            result["cpu_baseline"] = {"value": None, "error": str(e)[-300:]}
    if samples:
        try:
            result["error_vs_oracle"] = errors_vs_oracle(samples[0], samples[1], dev)
        except Exception as e:
            result["error_vs_oracle"] = {"error": str(e)[-300:]}
    return result


def _pct(v, q):
    v = sorted(v)
    return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))] if v else None


def bench_powerlaw(args, dev, world):
    """Chung-Lu power-law graph (2^20 vertices, mean degree 16, exponent 2.5,
    largest component, weights uniform in (0, 1]): PCG with the MSP, mixed
    precision against plain FP64, one N(0,1) right-hand side per solve."""
    import numpy as np
    import torch

    import graphgen as gg
    import paper_2207_07847_gb300 as P
    t0 = time.perf_counter()
    g = gg.chung_lu(args.powerlaw_n, avg_deg=16.0, gamma=2.5, weights="uniform01", seed=4)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    h = P.lap_setup(g, prec="msp", mu=WORKLOAD["mu"], precision="mixed", seed=WORKLOAD["setup_seed"],
                    tol=WORKLOAD["tol"], maxit=20000)
    setup_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    x = torch.empty(g.n, dtype=torch.float64, device=dev)
    out = {"workload": f"chunglu_{args.powerlaw_n}_d16_g2.5_uniform01_MSP_mu0.8", "n": g.n,
           "nnz": P.lap_get_hierarchy_info(h)["nnz"], "gen_s": round(gen_s, 2), "setup_s": round(setup_s, 2)}
    # the matvec on hub rows: SELL slices plus chunked long rows, against the copy bandwidth
    deg = np.diff(np.asarray(g.row_ptr))
    peak, peak_kind = measured_peaks()
    spmv = {"max_degree": int(deg.max()), "mean_degree": round(float(deg.mean()), 2),
            "entries_in_rows_over_8x_mean": round(float(deg[deg > 8 * deg.mean()].sum() / deg.sum()), 4)}
    # the autotuned choice, then SELL + chunks and the merge-path CSR forced
    for label, hk in (("tuned", h), ("sell", None), ("merge", None)):
        if hk is None:
            hk = P.lap_setup(g, prec="msp", mu=WORKLOAD["mu"], precision="mixed", seed=WORKLOAD["setup_seed"],
                             spmv_tpr=-1 if label == "sell" else -2)
        for prec_name, prec_id in (("fp32", 1), ("fp64", 0)):
            ms_, by_ = P.lap_kernel_bench(hk, "spmv_L", prec_id, 20)
            spmv[f"{label}_{prec_name}"] = {"us_per_launch": round(ms_ * 1e3, 2), "bytes_per_launch": by_,
                                            "gbs": round(by_ / (ms_ * 1e-3) / 1e9, 1),
                                            "frac": round(by_ / (ms_ * 1e-3) / 1e9 / peak, 4),
                                            "peak_kind": peak_kind}
        if hk is not h:
            hk.close()
    out["spmv_L"] = spmv
    for precision in ("mixed", "fp64", "fgmres"):
        # "fgmres": the paper's outer method, flexible GMRES(30), FP64
        if precision == "fgmres":
            P.lap_update_options(h, precision="fp64", krylov="fgmres", restart=30)
        else:
            P.lap_update_options(h, precision=precision)
        bs = [torch.as_tensor(gg.rhs(g.n, seed=800 + i), device=dev) for i in range(4)]
        P.lap_pcg_solve(h, bs[0], x)                                 # warm-up
        ranks_barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [P.lap_pcg_solve(h, b, x) for b in bs[1:]]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        out[precision] = {"value": whole_job_rate(len(infos), world, ms), "unit": "solves/s",
                          "iterations": [i.iterations for i in infos],
                          "relres_max": max(i.relres for i in infos),
                          "failed": sum(1 for i in infos if i.status != 0)}
    h.close()
    return out


def bench_pegp_exact(args, dev, world):
    """The small workload solved the paper's way: 2D grid (64 x 64, 4-neighbour,
    weights uniform in [1, 2]) coarsened to <= 32 vertices, PEGP applied
    exactly (dense inverse of the scaled L_H, built on the device at setup),
    mu = 1/sqrt(n), all FP64, one N(0,1) right-hand side per solve.  Also the
    Lanczos estimate of kappa(L_H^+ L_Gt) and the dense matvec's rates: FP64
    is bound by the FP64 pipe (one FMA per 8-byte entry), FP32 by HBM."""
    import torch

    import graphgen as gg
    import paper_2207_07847_gb300 as P
    side = args.exact_side
    g = gg.grid2d(side, weights="uniform", lo=1.0, hi=2.0, seed=1)
    mu = 1.0 / math.sqrt(g.n)
    t0 = time.perf_counter()
    h = P.lap_setup(g, prec="pegp_exact", mu=mu, precision="mixed", seed=WORKLOAD["setup_seed"],
                    tol=WORKLOAD["tol"], maxit=1000)
    setup_s = time.perf_counter() - t0
    info_h = P.lap_get_hierarchy_info(h)
    P.lap_update_options(h, precision="fp64")
    stream = torch.cuda.current_stream()
    x = torch.empty(g.n, dtype=torch.float64, device=dev)
    bs = [torch.as_tensor(gg.rhs(g.n, seed=900 + i), device=dev) for i in range(23)]
    for b in bs[:3]:
        P.lap_pcg_solve(h, b, x)                                     # warm-up
    ranks_barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [P.lap_pcg_solve(h, b, x) for b in bs[3:]]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    k_l, lo_l, hi_l = P.lap_estimate_condition(h)
    nt = info_h["ntilde"]
    # the paper's outer method on the same system: flexible GMRES(30)
    P.lap_update_options(h, krylov="fgmres", restart=30)
    P.lap_pcg_solve(h, bs[0], x)
    torch.cuda.synchronize()
    e0.record(stream)
    ginfos = [P.lap_pcg_solve(h, b, x) for b in bs[3:13]]
    e1.record(stream)
    torch.cuda.synchronize()
    gms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    P.lap_update_options(h, krylov="cg")
    # stretch of H over T (Section 3.3), tr(L_T^+ L_H) by 32 Hutchinson samples
    t0 = time.perf_counter()
    sv = P.lap_estimate_stretch(h, samples=32, seed=1)
    stretch_s = time.perf_counter() - t0
    m64, b64 = P.lap_kernel_bench(h, "pegp_gemv", 0, 20)
    m32, b32 = P.lap_kernel_bench(h, "pegp_gemv", 1, 20)
    out = {"workload": f"grid2d_{side}x{side}_uniform[1,2]_PEGP_exact_mu1/sqrt(n)_fp64", "n": g.n,
           "ntilde": nt, "levels": info_h["levels"], "mu": mu, "setup_s": round(setup_s, 3),
           "value": whole_job_rate(len(infos), world, ms), "unit": "solves/s",
           "ms_per_solve": ms / len(infos),
           "iterations": [i.iterations for i in infos][:5],
           "relres_max": max(i.relres for i in infos),
           "failed": sum(1 for i in infos if i.status != 0),
           "lanczos": {"steps": k_l, "lambda_min": lo_l, "lambda_max": hi_l, "kappa": hi_l / lo_l},
           "stretch": {"trace_LTplus_LH": float(sv.mean()),
                       "std_error": float(sv.std(ddof=1) / math.sqrt(len(sv))), "samples": len(sv),
                       "seconds": round(stretch_s, 4)},
           "fgmres": {"value": whole_job_rate(len(ginfos), world, gms), "unit": "solves/s",
                      "iterations": [i.iterations for i in ginfos][:5],
                      "relres_max": max(i.relres for i in ginfos),
                      "failed": sum(1 for i in ginfos if i.status != 0)},
           "dense_matvec": {
               "fp64": {"us": round(m64 * 1e3, 2), "GB/s": round(b64 / (m64 * 1e-3) / 1e9, 1),
                        "bound": "alu", "TFLOP/s": round(2.0 * nt * nt / (m64 * 1e-3) / 1e12, 3),
                        "peak_TFLOP/s": FP64_ALU_PEAK_TFLOPS, "peak_kind": "nominal"},
               "fp32": {"us": round(m32 * 1e3, 2), "GB/s": round(b32 / (m32 * 1e-3) / 1e9, 1),
                        "bound": "hbm"}}}
    h.close()
    return out


def bench_batched(args, dev, world):
    """Many right-hand sides at once: an R-MAT graph (scale s, edge factor 16,
    a, b, c = 0.57, 0.19, 0.19, largest component, unit weights) with
    `batched_rhs` N(0,1) columns solved together by lap_pcg_solve_batched (MSP,
    mu = 0.8, FP32 SpMM and sweeps with per-column FP64 refinement), against
    the plain FP64 single-solve path on a few of the same columns."""
    import torch

    import graphgen as gg
    import paper_2207_07847_gb300 as P
    t0 = time.perf_counter()
    g = gg.rmat(args.batched_scale, 16, seed=5)
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    h = P.lap_setup(g, prec="msp", mu=WORKLOAD["mu"], precision="mixed", seed=WORKLOAD["setup_seed"],
                    tol=WORKLOAD["tol"], maxit=20000)
    setup_s = time.perf_counter() - t0
    k = args.batched_rhs
    gen = torch.Generator(device=dev)
    gen.manual_seed(500)
    B = torch.randn(k, g.n, dtype=torch.float64, device=dev, generator=gen)
    X = torch.empty_like(B)
    stream = torch.cuda.current_stream()
    st, infos = P.lap_pcg_solve_batched([h], [B], [X])          # warm-up (autotune, graphs)
    ranks_barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st, infos = P.lap_pcg_solve_batched([h], [B], [X])
    e1.record(stream)
    torch.cuda.synchronize()
    ranks_barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    bad = sum(1 for i in infos if i.status != 0)
    # the plain FP64 single-solve path on the first columns
    P.lap_update_options(h, precision="fp64")
    ks = min(4, k)
    x1 = torch.empty(g.n, dtype=torch.float64, device=dev)
    P.lap_pcg_solve(h, B[0], x1)                                # warm-up
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    single = [P.lap_pcg_solve(h, B[j], x1) for j in range(ks)]
    f1.record(stream)
    torch.cuda.synchronize()
    ms1 = max_over_ranks(f0.elapsed_time(f1), world, dev)
    info = P.lap_get_hierarchy_info(h)
    h.close()
    its = sorted(i.iterations for i in infos)
    return {"workload": f"rmat_s{args.batched_scale}_ef16_unit_{k}rhs_MSP_mu0.8",
            "n": g.n, "nnz": info["nnz"], "levels": info["levels"], "rhs": k,
            "precision": "mixed (FP32 SpMM/sweeps, FP64 per-column refinement)",
            "value": whole_job_rate(k, world, ms), "unit": "solves/s",
            "ms_per_batch": ms, "iterations": {"median": its[len(its) // 2], "max": its[-1]},
            "relres_max": max(i.relres for i in infos), "failed": bad,
            "plain_fp64_single": {"value": whole_job_rate(ks, world, ms1), "unit": "solves/s",
                                  "columns": ks,
                                  "iterations": [i.iterations for i in single]},
            "gen_s": round(gen_s, 2), "setup_s": round(setup_s, 2)}


def bench_group(args, dev, world):
    """Many graphs of uneven size at once: `group_graphs` graphs with vertex
    counts log-uniform in [2e2, 1e5] (2D and 3D grids, Chung-Lu with mean
    degree 8..32, random geometric graphs; weights log-uniform in [1e-2,
    1e2]), each with 1..16 N(0,1) right-hand sides, MSP (mu = 0.8), mixed
    precision: one solve group (one launch per PCG phase for all graphs)
    against the same graphs solved one after another by the batched path."""
    import numpy as np
    import torch

    import paper_2207_07847_gb300 as P
    rng = np.random.default_rng(23)
    G = args.group_graphs
    sizes = np.exp(rng.uniform(math.log(2e2), math.log(1e5), G))
    kinds = ["grid2d", "grid3d", "chung_lu", "rgg"]
    graphs = [_serving_graph(kinds[i % 4], sizes[i], rng, 600 + i) for i in range(G)]
    hs = [P.lap_setup(g, prec="msp", mu=WORKLOAD["mu"], precision="mixed", seed=WORKLOAD["setup_seed"],
                      tol=WORKLOAD["tol"], maxit=20000) for g in graphs]
    nr = rng.integers(1, 17, G)
    gen = torch.Generator(device=dev)
    gen.manual_seed(800)
    Bs = [torch.randn(int(nr[i]), graphs[i].n, dtype=torch.float64, device=dev, generator=gen) for i in range(G)]
    Xs = [torch.empty_like(b) for b in Bs]
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    grp = P.Group(hs)
    create_s = time.perf_counter() - t0

    def timed(fn):
        fn()                                            # warm-up (graphs, workspaces)
        ranks_barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ranks_barrier(world)
        return max_over_ranks(e0.elapsed_time(e1), world, dev), out

    ms_g, (st, infos) = timed(lambda: P.lap_pcg_solve_group(grp, Bs, Xs))

    def sequential():
        allinf = []
        for i in range(G):
            st_, inf_ = P.lap_pcg_solve_batched([hs[i]], [Bs[i]], [Xs[i]])
            allinf += inf_
        return allinf

    ms_s, inf_s = timed(sequential)
    rhs = int(nr.sum())
    its = sorted(i.iterations for i in infos)
    out = {"workload": f"group_{G}graphs_n2e2..1e5_msp_mixed", "graphs": G,
           "n_min": int(min(g.n for g in graphs)), "n_max": int(max(g.n for g in graphs)),
           "n_total": int(sum(g.n for g in graphs)), "rhs": rhs,
           "value": whole_job_rate(rhs, world, ms_g), "unit": "solves/s", "ms": ms_g,
           "launches": int(infos[0].kernel_launches) if infos else 0,
           "iterations": {"median": its[len(its) // 2], "max": its[-1]},
           "relres_max": max(i.relres for i in infos), "failed": sum(1 for i in infos if i.status != 0),
           "create_s": round(create_s, 3),
           "graph_after_graph": {"value": whole_job_rate(rhs, world, ms_s), "unit": "solves/s", "ms": ms_s,
                                 "launches": int(sum(i.kernel_launches for i in inf_s[:1]) if inf_s else 0),
                                 "relres_max": max(i.relres for i in inf_s),
                                 "failed": sum(1 for i in inf_s if i.status != 0)}}
    grp.close()
    for h in hs:
        h.close()
    return out


def sweep_inner(args, g, dev):
    """PEGP inner cap x inner tolerance at the workload: one mixed solve each
    after a warm-up, solves/s and iterations (chooses the headline's settings)."""
    import torch

    import graphgen as gg
    import paper_2207_07847_gb300 as P
    h = P.lap_setup(g, prec="pegp_inner", mu=WORKLOAD["mu"], precision="mixed", seed=WORKLOAD["setup_seed"],
                    tol=WORKLOAD["tol"], inner_tol=0.1, inner_maxit=12, maxit=30000)
    stream = torch.cuda.current_stream()
    x = torch.empty(g.n, dtype=torch.float64, device=dev)
    b0 = torch.as_tensor(gg.rhs(g.n, seed=100), device=dev)
    b1 = torch.as_tensor(gg.rhs(g.n, seed=101), device=dev)
    rows = []
    for cap in (6, 12, 24):
        for tol in (0.3, 0.1, 0.01):
            P.lap_update_options(h, inner_maxit=cap, inner_tol=tol)
            P.lap_pcg_solve(h, b0, x)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = P.lap_pcg_solve(h, b1, x)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            rows.append({"inner_maxit": cap, "inner_tol": tol, "solves_per_s": 1e3 / ms, "ms": ms,
                         "outer": info.iterations, "inner": info.inner_iterations, "relres": info.relres,
                         "status": info.status})
            print(f"[sweep] {rows[-1]}", file=sys.stderr, flush=True)
    h.close()
    return {"sweep_inner": rows, "workload": WORKLOAD["name"]}


def _serving_graph(kind, n, rng, seed):
    import graphgen as gg
    w = dict(weights="loguniform", lo=1e-2, hi=1e2, seed=seed)
    if kind == "grid2d":
        return gg.grid2d(max(8, int(round(n ** 0.5))), **w)
    if kind == "grid3d":
        return gg.grid3d(max(4, int(round(n ** (1.0 / 3.0)))), **w)
    if kind == "chung_lu":
        return gg.chung_lu(int(n), avg_deg=float(rng.integers(8, 33)), **w)
    return gg.rgg(int(n), avg_deg=10.0, **w)


def bench_handshake(args, dev, world):
    """The headline grid with the deterministic parallel matching variant
    (LAP_MATCH_HANDSHAKE, a change of the paper's coarsening): MSP and PEGP_inner,
    mixed precision, one timed solve each after one warm-up, iterations beside
    the paper's matching.  Reported apart from the headline."""
    import torch

    import graphgen as gg
    import paper_2207_07847_gb300 as P
    g = gg.grid3d(args.nx, weights="loguniform", lo=WORKLOAD["wlo"], hi=WORKLOAD["whi"],
                  seed=WORKLOAD["wseed"])
    stream = torch.cuda.current_stream()
    x = torch.empty(g.n, dtype=torch.float64, device=dev)
    bs = [torch.as_tensor(gg.rhs(g.n, seed=950 + i), device=dev) for i in range(2)]
    out = {"workload": f"grid3d_{args.nx}^3_loguniform, matching = handshake",
           "setup": "setup_s: lap_setup with the hierarchy and L_H built on the host threads; "
                    "setup_device_s: the same setup with them built by device kernels "
                    "(setup_device = 1, bit-exact with the host build); the solves use the latter"}
    for prec in ("msp", "pegp_inner"):
        kw = dict(prec=prec, mu=WORKLOAD["mu"], precision="mixed", matching="handshake",
                  tol=WORKLOAD["tol"], inner_tol=WORKLOAD["inner_tol"],
                  inner_maxit=WORKLOAD["inner_maxit"], maxit=30000, timeout_s=120.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = P.lap_setup(g, **kw)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        h.close()
        t0 = time.perf_counter()
        h = P.lap_setup(g, setup_device=1, **kw)
        torch.cuda.synchronize()
        setup_device_s = time.perf_counter() - t0
        P.lap_pcg_solve(h, bs[0], x)                              # warm-up
        ranks_barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = P.lap_pcg_solve(h, bs[1], x)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        out[prec] = {"value": whole_job_rate(1, world, ms), "unit": "solves/s",
                     "levels": P.lap_get_hierarchy_info(h)["levels"], "setup_s": round(setup_s, 2),
                     "setup_device_s": round(setup_device_s, 2),
                     "iterations": info.iterations, "inner_iterations": info.inner_iterations,
                     "relres": info.relres, "status": info.status}
        h.close()
    return out


def bench_serving(args, dev, world):
    """Continuous-batching server: `serve_graphs` resident graphs with vertex
    counts log-uniform in [1e3, serve_nmax] (2D and 3D grids, Chung-Lu with
    mean degree 8..32, random geometric graphs; weights log-uniform in
    [1e-2, 1e2]), `serve_requests` requests of 1..16 N(0,1) right-hand sides
    arriving as a Poisson stream at half the server's measured capacity
    (MSP, mu = 0.8, relres 1e-8; FP32 columns refined per request in FP64).
    The same stream (a prefix of it, within a time limit) through the plain
    FP64 single-solve path for comparison."""
    import numpy as np
    import torch

    import paper_2207_07847_gb300 as P
    rng = np.random.default_rng(11)
    G = args.serve_graphs
    sizes = np.exp(rng.uniform(math.log(1e3), math.log(args.serve_nmax), G))
    kinds = ["grid2d", "grid3d", "chung_lu", "rgg"]
    t0 = time.perf_counter()
    graphs = [_serving_graph(kinds[i % 4], sizes[i], rng, 300 + i) for i in range(G)]
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    hs = [P.lap_setup(g, prec="msp", mu=WORKLOAD["mu"], precision="mixed", seed=WORKLOAD["setup_seed"],
                      tol=WORKLOAD["tol"], maxit=20000) for g in graphs]
    setup_s = time.perf_counter() - t0
    R = args.serve_requests
    gi = rng.integers(0, G, R)
    nr = rng.integers(1, 17, R)
    gen = torch.Generator(device=dev)
    gen.manual_seed(700)
    Bs = [torch.randn(int(nr[i]), graphs[gi[i]].n, dtype=torch.float64, device=dev, generator=gen)
          for i in range(R)]
    Xs = [torch.empty_like(b) for b in Bs]
    S = P.Server(max_slots=16, check_every=8, hbm_budget_bytes=96 << 30)

    def run_stream(idx, arrivals):
        """Submit requests idx at the given offsets (s); returns per-request
        (latency s, status) and the wall time from first arrival to last completion."""
        done = {}
        ids = []
        start = time.perf_counter()
        for j, i in enumerate(idx):
            delay = start + arrivals[j] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids.append((i, time.perf_counter(), S.submit(hs[gi[i]], Bs[i], Xs[i])))
        last = start
        for i, t_sub, rid in ids:
            st, info = S.wait(rid, 600.0)
            done[i] = (info.seconds, st, info.as_dict())
            last = max(last, t_sub + info.seconds)
        return done, last - start

    # capacity: a closed burst of the first requests (all submitted at once)
    burst = list(range(min(256, R)))
    _, t_burst = run_stream(burst, [0.0] * len(burst))
    cap_rhs = float(sum(nr[i] for i in burst)) / t_burst
    lam = args.serve_load * cap_rhs / float(np.mean(nr))     # requests per second
    print(f"serving: burst of {len(burst)} requests in {t_burst:.1f} s ({cap_rhs:.1f} RHS/s)",
          file=sys.stderr, flush=True)
    arrivals = np.cumsum(rng.exponential(1.0 / lam, R))
    arrivals -= arrivals[0]
    ranks_barrier(world)
    done, wall = run_stream(list(range(R)), arrivals)
    S.close()
    print(f"serving: {R} requests in {wall:.1f} s", file=sys.stderr, flush=True)
    lat = [done[i][0] * 1e3 for i in range(R)]
    failed = sum(1 for i in range(R) if done[i][1] != 0)
    failed_info = [dict(done[i][2], graph_n=graphs[gi[i]].n, nrhs=int(nr[i]))
                   for i in range(R) if done[i][1] != 0][:5]
    restarted = sum(1 for i in range(R) if done[i][2].get("restarts", 0) > 0)
    rhs_total = int(nr.sum())
    wall = max_over_ranks(wall, world, dev)
    # plain FP64 single solves of the same stream (prefix), FIFO, real time
    for h in hs:
        P.lap_update_options(h, precision="fp64")
    plain_lat, plain_rhs = [], 0
    x1 = {}
    start = time.perf_counter()
    for i in range(R):
        now = time.perf_counter() - start
        if now > args.serve_plain_s:
            break
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        g = graphs[gi[i]]
        if g.n not in x1:
            x1[g.n] = torch.empty(g.n, dtype=torch.float64, device=dev)
        for j in range(int(nr[i])):
            P.lap_pcg_solve(hs[gi[i]], Bs[i][j], x1[g.n])
        torch.cuda.synchronize()
        plain_lat.append((time.perf_counter() - start - arrivals[i]) * 1e3)
        plain_rhs += int(nr[i])
    plain_wall = time.perf_counter() - start
    for h in hs:
        h.close()
    K = len(plain_lat)
    lat_prefix = lat[:K]
    rhs_prefix = int(nr[:K].sum())
    return {"workload": f"serving_{G}graphs_n1e3..{args.serve_nmax:.0e}_{R}req_poisson",
            "graphs": {"count": G, "n_min": int(min(g.n for g in graphs)),
                       "n_max": int(max(g.n for g in graphs)), "kinds": kinds},
            "requests": R, "rhs_total": rhs_total, "arrival_rate_req_s": round(lam, 2),
            "capacity_rhs_s": round(cap_rhs, 1), "load": args.serve_load,
            "arrivals": f"Poisson at {args.serve_load} x the capacity of a closed burst of the "
                        f"first {len(burst)} requests",
            "precision": "mixed (FP32 columns refined per request in FP64), 16 per graph batch",
            "value": whole_job_rate(rhs_total, world, wall * 1e3),
            "unit": "solves/s", "requests_per_s": R * world / wall,
            "latency_ms": {"p50": _pct(lat, 0.5), "p99": _pct(lat, 0.99)}, "failed": failed,
            "failed_info": failed_info, "restarted_requests": restarted,
            "plain_fp64_single": {"requests": K, "rhs": plain_rhs,
                                  "value": plain_rhs / plain_wall, "unit": "solves/s",
                                  "latency_ms": {"p50": _pct(plain_lat, 0.5),
                                                 "p99": _pct(plain_lat, 0.99)},
                                  "time_limit_s": args.serve_plain_s,
                                  "stream": "the server's first requests, same arrival times, "
                                            "FIFO single solves"},
            "server_on_plain_prefix": {"requests": K, "rhs": rhs_prefix,
                                       "latency_ms": {"p50": _pct(lat_prefix, 0.5),
                                                      "p99": _pct(lat_prefix, 0.99)}},
            "gen_s": round(gen_s, 2), "setup_s": round(setup_s, 2)}


def bench_reference(args):
    """The oracle as the reference arm, by the same method as the cpu_baseline
    leg: its PCG on the full workload (setup excluded), timed over the outer
    iterations that fit args.oracle_cap_s seconds after args.warmup untimed
    ones, single-threaded; solves/s = 1 / (seconds per outer iteration x
    REF_OUTER_ITERATIONS).  A step is one outer iteration."""
    cap = args.oracle_cap_s
    proc = start_oracle(args.nx, args.prec, cap, 1, False)
    rep = finish_oracle(proc)
    rate, per_iter = oracle_rate(rep, REF_OUTER_ITERATIONS)
    hd = host_description()
    sample = (f"oracle (numpy/scipy PCG with the PEGP inner solve, 1 thread) on the full {rep['n']}-vertex "
              f"workload, setup excluded ({rep['setup_s']:.0f} s): {rep['outer']} outer ({rep['inner']} inner) "
              f"iterations in {rep['seconds']:.1f} s; solves/s = 1 / (s per outer iteration x "
              f"{REF_OUTER_ITERATIONS} outer iterations per solve)")
    return {"metric": METRIC, "value": rate, "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_iter,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD["name"] if args.nx == 128 else f"grid3d_{args.nx}^3",
                       "step": (f"one outer PCG iteration of the oracle ({WORKLOAD['inner_maxit']} inner "
                                f"iterations); the timed region holds the {rep['outer']} that fit "
                                f"{cap:.0f} s"),
                       "host": hd},
            "cpu_baseline": {"value": rate, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.oracle_worker:
        oracle_worker(args.oracle_worker)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(bench_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    if args.serving_only:
        args.only = "serving"
    if args.only:
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        line = {"serving": bench_serving, "powerlaw": bench_powerlaw, "batched": bench_batched,
                "group": bench_group, "handshake": bench_handshake, "pegp_exact": bench_pegp_exact}[args.only]
        res = {args.only: line(args, dev, world)}
        if rank == 0:
            print(json.dumps(res), flush=True)
        return
    res = bench_ours(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
