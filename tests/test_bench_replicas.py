"""The N > 1 path of bench.py on the CPU: ranks are replicas (no collective on
the data path), the job's time is the slowest rank's, the whole-job rate
counts every rank's units, and only rank 0 runs and prints the reference arm.
Two gloo processes stand in for two GPUs."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        bench.ranks_barrier(world)
        ms = 10.0 * (rank + 1)                       # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, world)
        rate = bench.whole_job_rate(3, world, ms_max)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ms_max": ms_max, "rate": rate}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["ms_max"] == 20.0
        assert r["rate"] == pytest.approx(3 * 2 / 0.020)


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_rate(4, 1, 500.0) == pytest.approx(8.0)
    bench.ranks_barrier(1)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"],
                         capture_output=True, text=True, env=env, timeout=120)
    assert out.returncode == 0
    assert out.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference on one rank: one JSON line with the contract's
    keys, the oracle as the reference, its own value as e2e with no copies."""
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    # a small instance of the workload's generator and a short timed region
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--nx", "14", "--oracle-cap-s", "1"],
                         capture_output=True, text=True, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    r = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in r, k
    assert r["impl"] == "reference" and r["steps"] == 1 and r["n_gpus"] == 1
    assert r["value"] > 0 and r["higher_is_better"] is True
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"] and cb["sample"]
    assert r["config"]["host"]["nproc"] >= 1 and r["config"]["host"]["cpu_model"]
    e = r["e2e"]
    assert e["value"] == r["value"] and e["unit"] == r["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
