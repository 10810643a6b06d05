"""Multi-rank host logic of bench.py on the CPU: two gloo ranks (replicas, no GPU).

Every rank times its own copy of the work; the job's time is the slowest rank's (every
rank gets the maximum), the job's rate counts the units of all ranks, and only rank 0 of
the reference arm does any work.
"""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), BENCH_GLOO="1")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    w, r, _ = bench.dist_setup()
    local_ms = [120.0, 300.0][r]
    ms = bench.max_over_ranks(local_ms, w)
    rate = bench.job_throughput(64 * 10, w, ms)
    dist.barrier()
    with open(os.path.join(out_dir, f"r{r}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "ms": ms, "rate": rate}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["world"] == 2 and r["ms"] == 300.0
        assert r["rate"] == pytest.approx(2 * 640 / 0.3)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(640, 1, 250.0) == pytest.approx(2560.0)


def test_reference_arm_other_ranks_do_nothing(capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    bench.run_reference(argparse.Namespace(workload="small", steps=1, warmup=0), 2, 1)
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the CPU oracle and prints one JSON line with the
    same metric, unit and direction as the GPU arm, plus its own cpu_baseline and e2e."""
    import subprocess

    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "small", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench

    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "iter/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "iter/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_kernel_source_hash_ignores_comments():
    """The DRAM traffic recorded from ncu is keyed to the kernels' code: comments and blank
    lines do not change the key, code does."""
    import bench

    a = "int f(int x) {  // one\n  /* two\n three */ return x + 1;\n\n}\n"
    b = "int f(int x) {\n  return x + 1;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(b.replace("+ 1", "+ 2"))
    assert len(bench.kernel_source_hash()) == 16


def test_error_vs_fp64_definitions():
    """The mixed-precision error report: relative 2-norm distances of x and y from the FP64
    answer, and each objective's error against p* relative to 1 + |p*|."""
    import numpy as np

    import bench

    fp64 = (np.array([3.0, 4.0]), np.array([1.0, 0.0]), -10.0)
    same = bench.error_vs_fp64(fp64, fp64, -10.0)
    assert same == {"x_rel": 0.0, "y_rel": 0.0, "obj_p_err_mixed": 0.0, "obj_p_err_fp64": 0.0}
    mixed = (np.array([3.0, 4.5]), np.array([1.0, 0.0]), -9.0)
    r = bench.error_vs_fp64(mixed, fp64, -10.5)
    assert r["x_rel"] == 0.5 / 5.0 and r["y_rel"] == 0.0
    assert r["obj_p_err_mixed"] == 1.5 / 11.5 and r["obj_p_err_fp64"] == 0.5 / 11.5
