#!/usr/bin/env python
"""Benchmark of the single-GPU PDHG hot path (one JSON line on stdout).

Workload: the power-law LP (n = 4,000,000 variables, m = 2,000,000 rows, ~40M nonzeros,
Pareto row lengths capped at 100k, seed 1), FP64.  One step = one body of the solver's CUDA
graph: 64 fused PDHG iterations (primal kernel + dual kernel each) and one check (KKT,
fixed-point residual, restart, PID).  ``value`` is PDHG iterations per second with the LP
resident in HBM; ``e2e`` is the same metric through the C ABI with host buffers (pinned):
each step uploads the start point, runs 64 iterations from it and reads the solution back.

``batch`` (default run): 256 uneven LPs solved together in one handle against the same LPs
solved one after another (time to 1e-4), plus the batch's iteration throughput.

``--impl reference`` times the CPU oracle on the same workload and metric (one PDHG
iteration per step, on the host cores).  With torchrun (N > 1) every rank solves its own
copy (replicas, no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import re
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 rel. KKT & PDHG iters/s; SpMV HBM GB/s vs peak; plain vs chosen form"
WORKLOAD = "powerlaw LP n=4,000,000 m=2,000,000 nnz~40M (Pareto-1.5 rows capped 100k, seed 1), FP64"
K_CHECK = 64
FP64_FMA_PER_CLK_SM = 2  # GB300 FP64 issue rate (measured: 1.90 FMA/clk/SM)
N_SM = 152


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="powerlaw", choices=["powerlaw", "powerlaw_quarter", "small"])
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--tol-runs", default="default", choices=["none", "small", "default", "all"],
                   help="time-to-tolerance runs: default = small LP to 1e-4 and 1e-8 and the "
                        "benchmark LP to 1e-4 (FP64 and mixed precision); all adds the "
                        "benchmark LP to 1e-8; small = only the small and tiny LPs; none")
    p.add_argument("--cpu-sample-iters", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the batched form (256 uneven LPs solved together vs one by one)")
    p.add_argument("--batch-count", type=int, default=256)
    p.add_argument("--batch-tols", default="1e-4,1e-6",
                   help="tolerances of the batched-vs-sequential comparison (1e-8: several "
                        "minutes; a few of the 256 LPs need more than 10^6 iterations)")
    p.add_argument("--batch-precond", type=int, default=0, choices=[0, 1])
    p.add_argument("--batch-tol8-count", type=int, default=64,
                   help="the smallest instances of the batch solved to 1e-8, batched and one by one")
    p.add_argument("--no-warm-start", action="store_true",
                   help="skip the learned warm start (train on solver solutions, warm vs cold)")
    p.add_argument("--ws-train", type=int, default=400,
                   help="warm start: training instances of the transportation family")
    p.add_argument("--ws-test", type=int, default=32, help="warm start: held-out instances")
    p.add_argument("--ws-epochs", type=int, default=8, help="warm start: training epochs")
    p.add_argument("--gnn-only", type=int, default=0, metavar="N",
                   help="time N training steps of the warm-start network on the transportation "
                        "family's graph (seeded targets) and exit: one JSON line of its own "
                        "(for profiling the network's kernels)")
    p.add_argument("--x3-full", action="store_true",
                   help="learned warm start with 2,000 training and 200 held-out instances of "
                        "the transportation family (default: --ws-train / --ws-test); several minutes")
    p.add_argument("--host-loop", action="store_true",
                   help="launch the iteration kernels from a host loop instead of the CUDA graph "
                        "(same kernels; for profilers that do not descend into graph loops)")
    return p.parse_args()


def make_lp(workload):
    import lpgen

    if workload == "powerlaw":
        return lpgen.powerlaw_lp(1)
    if workload == "powerlaw_quarter":  # same recipe at 1/4 size, for profiler captures
        return lpgen.scaled_powerlaw_lp(1, 0.25)
    return lpgen.small_random_lp(0)


def workload_name(workload):
    if workload == "powerlaw":
        return WORKLOAD
    if workload == "powerlaw_quarter":
        return "powerlaw LP at 1/4 size: n=1,000,000 m=500,000 nnz~10M (cap 50k, seed 1), FP64"
    return "small random LP n=2,000 m=1,000 (600 '=', 400 '<='), 16,000 nnz, seed 0, FP64"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _code_only(text):
    """C++ source without comments, blank lines and whitespace differences (string literals
    are left alone: the kernel sources hold no comment markers inside them)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    lines = (" ".join(re.sub(r"//.*", "", line).split()) for line in text.splitlines())
    return "\n".join(line for line in lines if line)


def kernel_source_hash():
    """Hash of the kernels' code (comments and blank lines ignored): the recorded DRAM
    traffic is used only while it matches."""
    h = hashlib.sha256()
    for f in ("kernels.cu", "internal.h"):
        with open(os.path.join(ROOT, "paper_2601_07628_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic_powerlaw_4Mx2M.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        if "=" in ln and not ln.startswith("#"):
            k, v = ln.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    v = kv.get(f"{kernel}_dram_bytes_per_launch")
    return float(v) if v else None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = sorted(float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit())
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4)
                          if r[5 + i].strip() == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx[0] if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline_subprocess(workload, iters):
    """Time the CPU oracle on a bounded sample (``iters`` PDHG iterations of the same LP) in a
    spawned process (no fork after CUDA init): once on one thread, once with its two sparse
    products split over every host core by row blocks (``oracle.rowsplit``, bitwise the same
    iterates).  The all-core figure is the line's value; the one-thread figure sits beside it."""
    code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
import bench
from oracle import pdhg as O
from oracle.rowsplit import RowSplitLP
lp = bench.make_lp({workload!r})
base = O.OracleLP.from_lpgen(lp)
eta = 1.0 / float(np.linalg.norm(lp.val))
res = {{}}
for threads, k in ((1, {iters}), (os.cpu_count() or 1, 2 * {iters})):
    o = RowSplitLP(base, threads)
    st = O.solve(o, eps=0.0, max_iter=1, params=dict(eta=eta)).state
    t0 = time.perf_counter()
    r = O.solve(o, eps=0.0, max_iter=1 + k, params=dict(eta=eta), state=st)
    res[threads] = dict(iters=k, seconds=time.perf_counter() - t0)
    o.close()
print(json.dumps(res))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                         timeout=1800)
    if out.returncode != 0:
        return {"value": None, "unit": "iter/s", "cores": 1, "kind": "oracle",
                "sample": "failed: " + out.stderr.strip().splitlines()[-1] if out.stderr else "failed"}
    d = {int(k): v for k, v in json.loads(out.stdout.strip().splitlines()[-1]).items()}
    many = max(d)
    one = d[1]
    return {"value": d[many]["iters"] / d[many]["seconds"], "unit": "iter/s", "cores": many,
            "kind": "oracle",
            "sample": f"{d[many]['iters']} oracle PDHG iterations (no check among them) of the same "
                      f"LP in {d[many]['seconds']:.1f} s; sparse products split over {many} host "
                      f"threads by row blocks (bitwise the one-thread iterates), vector updates "
                      f"on one thread",
            "single_thread": {"value": one["iters"] / one["seconds"], "unit": "iter/s", "cores": 1,
                              "sample": f"{one['iters']} iterations in {one['seconds']:.1f} s"}}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if os.environ.get("BENCH_GLOO") is None else "gloo")
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    """The largest value over all ranks (every rank gets it); the identity for one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


def cusparse_reference(lp, dev, kb, reps=30):
    """CUDA-event time of torch's CSR matrix-vector product (cuSPARSE SpMV) for A x and A^T y
    on the LP's matrix (FP64 values, int32 indices), with the bytes of the product alone
    (12 per nonzero + row pointers + the gathered and written vectors)."""
    import numpy as np
    import scipy.sparse as sp
    import torch

    d = f"cuda:{dev}"
    A = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
    At = A.T.tocsr()
    out = {}
    for name, M, nin in (("A_x", A, lp.n), ("AT_y", At, lp.m)):
        T = torch.sparse_csr_tensor(torch.from_numpy(M.indptr.astype(np.int32)).to(d),
                                    torch.from_numpy(M.indices.astype(np.int32)).to(d),
                                    torch.from_numpy(M.data).to(d), size=M.shape, dtype=torch.float64)
        v = torch.rand(nin, 1, dtype=torch.float64, device=d)
        for _ in range(3):
            T @ v
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            T @ v
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        by = 12 * M.nnz + 4 * (M.shape[0] + 1) + 8 * nin + 8 * M.shape[0]
        out[name] = {"ms": ms, "GB/s": by / (ms * 1e-3) / 1e9}
        del T, v
    torch.cuda.empty_cache()
    out["note"] = ("torch.sparse_csr_tensor @ dense (cuSPARSE SpMV); the solver's primal / dual "
                   "kernels compute A^T y / A x_bar plus the whole primal / dual step")
    return out


def run_gnn_only(args, dev):
    """The warm-start network's training step alone: ``--gnn-only`` captured steps
    (``dpdlp_gnn_train_step``: features, forward, backward, Adam) on the 300 x 300
    transportation family's graph, two instances alternating, seeded random targets, after
    3 untimed steps."""
    import numpy as np
    import torch

    import lpgen
    from paper_2601_07628_gb300 import gnn

    fam = lpgen.transport_family(seed=4)
    lps = [lpgen.transport_lp(fam, 100 + i) for i in range(2)]
    rng = np.random.default_rng(0)
    xs = [rng.random(lp.n) for lp in lps]
    ys = [rng.standard_normal(lp.m) for lp in lps]
    sc = gnn.fit_scales(lps, xs, ys)
    net = gnn.Network(dev)
    net.set_params(gnn.init_params(0))
    net.set_graph(lps[0].n, lps[0].m, lps[0].row_ptr, lps[0].col, lps[0].val)
    net.device_arrays(True)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(f"cuda:{dev}")
    data = [(t(fv), t(fc), t(x / sc.x_scale), t(y / sc.y_scale))
            for lp, x, y in zip(lps, xs, ys) for fv, fc in [gnn.features(lp, sc)]]
    for step in range(1, 4):
        net.train_step(*data[step % 2], 1e-3, step)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for step in range(4, 4 + args.gnn_only):
        net.train_step(*data[step % 2], 1e-3, step, want_loss=False)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / max(args.gnn_only, 1)
    net.close()
    print(json.dumps({"gnn_train_step_ms": ms, "steps": args.gnn_only,
                      "graph": f"transportation 300 x 300 + 20000 side rows (n={lps[0].n:,}, "
                               f"m={lps[0].m:,}, nnz={lps[0].nnz:,})"}), flush=True)


def run_reference(args, world, rank):
    """The CPU oracle on the same workload and metric: a step is one PDHG iteration of one
    continuing oracle solve.  The K timed steps run inside one solve call, so the oracle
    checks at its own cadence (every 64 iterations, and once when the call ends) instead of
    once per step."""
    if rank != 0:
        return
    import numpy as np

    from oracle import pdhg as O

    from oracle.rowsplit import RowSplitLP

    lp = make_lp(args.workload)
    cores = os.cpu_count() or 1
    o = RowSplitLP(O.OracleLP.from_lpgen(lp), cores)  # products on every host core
    eta = 1.0 / float(np.linalg.norm(lp.val))
    params = dict(eta=eta)
    st = O.solve(o, eps=0.0, max_iter=0, params=params).state
    st = O.solve(o, eps=0.0, max_iter=args.warmup, params=params, state=st).state
    t0 = time.perf_counter()
    r = O.solve(o, eps=0.0, max_iter=args.warmup + args.steps, params=params, state=st)
    dt = time.perf_counter() - t0
    checks = len(r.trace)
    v = args.steps / dt
    o.close()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.workload),
                       "step": "1 PDHG iteration of the CPU oracle (numpy/scipy FP64)",
                       "parallelism": "host"},
            "cpu_baseline": {"value": v, "unit": "iter/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} consecutive oracle PDHG iterations of one "
                                       f"solve ({checks} checks among them: every 64 iterations "
                                       f"and at the end) after {args.warmup} warm-up iterations; "
                                       f"sparse products split over {cores} host threads by row "
                                       f"blocks (bitwise the one-thread iterates)"},
            "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_to_tol(s, tol, max_iter, fp32_mode=0):
    """Fresh solve to ``tol`` from the default start (x = proj_X(0), y = 0) on a loaded
    handle (power iteration and graph build done by a 64-iteration solve before the timed
    one).  A start point set earlier on the handle stays set until cleared, so it is
    cleared here."""
    s.set_start(None, None)
    s.set_param("resume", 0)
    s.set_param("spmv_fp32", fp32_mode)
    s.solve(tol, 64)
    t0 = time.perf_counter()
    st = s.solve(tol, max_iter)
    dt = time.perf_counter() - t0
    k = s.kkt()
    tr = s.trace(1 << 16)
    switch = next((r["T"] for r in tr if r["spmv_mode"] == 0), None) if fp32_mode else None
    return {"tol": tol, "form": ["fp64", "mixed_fp32", "fp32_values"][fp32_mode], "status": st,
            "precond": int(s.get_param("precond")),
            "seconds": dt, "iterations": k["iterations"], "restarts": k["restarts"],
            "rel_kkt": max(k["r_primal"], k["r_dual"], k["r_gap"]),
            "fp64_from_iteration": switch}


def solution_and_objective(s):
    import numpy as np

    x, y = s.solution()
    return np.array(x, copy=True), np.array(y, copy=True), s.kkt()["obj_p"]


def error_vs_fp64(mixed, fp64, p_star):
    """How far a mixed-precision answer lies from the FP64 answer to the same tolerance
    (the FP64 path is the one that matches the oracle iterate for iterate): relative
    2-norm distances of x and y, and each objective's error against the planted optimum
    value p*, relative to 1 + |p*|."""
    import numpy as np

    def rel(a, b):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    return {"x_rel": rel(mixed[0], fp64[0]), "y_rel": rel(mixed[1], fp64[1]),
            "obj_p_err_mixed": abs(mixed[2] - p_star) / (1.0 + abs(p_star)),
            "obj_p_err_fp64": abs(fp64[2] - p_star) / (1.0 + abs(p_star))}


def _uneven(args):
    import lpgen

    return lpgen.uneven_lp(*args)


def make_batch(count, seed=3):
    """The batched workload (``lpgen.batch_lps``), instances generated in a process pool
    started with spawn."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    import lpgen

    ms = lpgen.batch_sizes(seed, count)
    jobs = [(1000 * seed + i, int(mi)) for i, mi in enumerate(ms)]
    workers = max(1, min(16, os.cpu_count() or 1))
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_uneven, jobs, chunksize=4))


def launches_per_body(info, ninst):
    """Kernel launches of one graph body (K iterations and one check)."""
    lr, lc = int(info["long_rows"] > 0), int(info["long_cols"] > 0)
    it = (1 + lc) + (1 + lr)
    check = (1 + lr) + (1 + lc) + int(info["m"] > 0) + int(info["n"] > 0) + 2 + 1
    return K_CHECK * it + check


def run_batch(args, dev, stream, peak):
    """Batched form: the LPs in one handle (per-instance step sizes, weights, restarts and
    statuses; converged instances are skipped), against the same LPs solved one after
    another with the single-LP path (``--batch-precond``: both preconditioned).  Power
    iteration and graph
    capture happen in an untimed 64-iteration solve before each timed solve, on both
    sides."""
    import numpy as np
    import torch

    from paper_2601_07628_gb300 import autotune
    from paper_2601_07628_gb300.costmodel import kernel_bytes
    from paper_2601_07628_gb300.dpdlp import Solver

    t0 = time.perf_counter()
    lps = make_batch(args.batch_count)
    gen_s = time.perf_counter() - t0
    n = sum(lp.n for lp in lps)
    m = sum(lp.m for lp in lps)
    nnz = sum(lp.nnz for lp in lps)
    s = Solver(dev)
    s.set_stream(stream)
    s.set_param("precond", args.batch_precond)
    t0 = time.perf_counter()
    s.load_batch(lps)
    load_s = time.perf_counter() - t0
    info = s.info()
    tune = autotune.tune(s, cache=os.path.join(tempfile.gettempdir(), "dpdlp_autotune.json"),
                         reps=10, rounds=2, force=True)
    # throughput with every instance running (fixed iteration counts, no convergence)
    s.set_param("resume", 1)
    T = 0
    for _ in range(3):
        T += K_CHECK
        s.solve(0.0, T)
    torch.cuda.synchronize()
    steps = max(3, args.steps // 10)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        T += K_CHECK
        s.solve(0.0, T)
    e1.record()
    torch.cuda.synchronize()
    it_s = steps * K_CHECK / (e0.elapsed_time(e1) / 1e3)
    kb = kernel_bytes(n, m, nnz)
    kt = {k: s.time_kernel(k, 20) for k in ("primal", "dual")}
    kern = {k: {"ms": kt[k], "GB/s": kb[k] / (kt[k] * 1e-3) / 1e9,
                "hbm_frac": kb[k] / (kt[k] * 1e-3) / 1e9 / peak} for k in kt}
    # batched solves to tolerance, then the same LPs one by one (plain FP64 PDHG)
    tols = sorted({float(t) for t in args.batch_tols.split(",")}, reverse=True)
    res_tol = {}
    for tol in tols:
        s.set_param("resume", 0)
        s.solve(tol, K_CHECK)
        t0 = time.perf_counter()
        st = s.solve(tol, 1_000_000)
        batched_s = time.perf_counter() - t0
        bk = s.batch_kkt()
        iters = np.array([k["iterations"] for k in bk], dtype=np.float64)
        res_tol[tol] = dict(batched_s=batched_s, st=st, iters=iters,
                            conv=int(sum(k["status"] == 0 for k in bk)))
    s.close()
    one = Solver(dev)
    one.set_stream(stream)
    one.set_param("precond", args.batch_precond)
    seq = {tol: dict(s=0.0, iters=[], status=[]) for tol in tols}
    seq_load = 0.0
    for lp in lps:
        t0 = time.perf_counter()
        one.load(lp)
        seq_load += time.perf_counter() - t0
        for tol in tols:
            r = time_to_tol(one, tol, 1_000_000, 0)
            seq[tol]["s"] += r["seconds"]
            seq[tol]["iters"].append(r["iterations"])
            seq[tol]["status"].append(r["status"])
    one.close()
    per_tol = {}
    for tol in tols:
        R, Q = res_tol[tol], seq[tol]
        per_tol[f"{tol:.0e}"] = {
            "batched": {"seconds": R["batched_s"], "status": R["st"], "converged": R["conv"],
                        "max_iterations": int(R["iters"].max()),
                        "sgm10_iterations": float(np.exp(np.mean(np.log(R["iters"] + 10.0))) - 10.0)},
            "sequential": {"seconds": Q["s"], "converged": int(sum(x == 0 for x in Q["status"])),
                           "max_iterations": int(max(Q["iters"]))},
            "speedup_vs_sequential": Q["s"] / R["batched_s"] if R["batched_s"] > 0 else None}
    return {
        "workload": f"{len(lps)} uneven LPs (m_i ~ U{{500..50000}}, n_i = 2 m_i, 5-15 nnz/col, seed 3): "
                    f"n={n:,} m={m:,} nnz={nnz:,}",
        "generate_s": gen_s, "load_s": load_s, "preprocess_ms": info["preprocess_ms"],
        "autotune": {k: tune[k] for k in ("cta_slots_primal", "cta_slots_dual", "list_fraction",
                                          "list_warps_per_sm", "ms") if k in tune},
        "iter_per_s_all_running": it_s, "kernels": kern,
        "gpu_launches_per_body": launches_per_body(info, len(lps)),
        "precond": args.batch_precond, "sequential_load_s": seq_load, "to_tol": per_tol,
        "to_1e-08_smallest": batch_tol8_smallest(args, lps, dev, stream),
    }


def batch_tol8_smallest(args, lps, dev, stream):
    """Relative KKT 1e-8 for the ``--batch-tol8-count`` smallest instances of the batch
    workload: batched (tuned launch choices) against the same LPs solved one after another."""
    import numpy as np

    from paper_2601_07628_gb300 import autotune
    from paper_2601_07628_gb300.dpdlp import Solver

    k = min(args.batch_tol8_count, len(lps))
    if k <= 0:
        return None
    pick = sorted(range(len(lps)), key=lambda i: (lps[i].nnz, i))[:k]
    sub = [lps[i] for i in pick]
    s = Solver(dev)
    s.set_stream(stream)
    s.load_batch(sub)
    tune = autotune.tune(s, cache=os.path.join(tempfile.gettempdir(), "dpdlp_autotune.json"),
                         reps=10, rounds=2, force=True)
    s.solve(1e-8, K_CHECK)
    s.set_param("resume", 0)
    t0 = time.perf_counter()
    st = s.solve(1e-8, 2_000_000)
    bs = time.perf_counter() - t0
    bk = s.batch_kkt()
    s.close()
    one = Solver(dev)
    one.set_stream(stream)
    seq_s, seq_it, seq_st = 0.0, [], []
    for lp in sub:
        one.load(lp)
        r = time_to_tol(one, 1e-8, 2_000_000, 0)
        seq_s += r["seconds"]
        seq_it.append(r["iterations"])
        seq_st.append(r["status"])
    one.close()
    it = np.array([q["iterations"] for q in bk], dtype=np.float64)
    return {"instances": k, "nnz": int(sum(lp.nnz for lp in sub)),
            "batched": {"seconds": bs, "status": st, "converged": int(sum(q["status"] == 0 for q in bk)),
                        "max_iterations": int(it.max())},
            "sequential": {"seconds": seq_s, "converged": int(sum(x == 0 for x in seq_st)),
                           "max_iterations": int(max(seq_it))},
            "speedup_vs_sequential": seq_s / bs if bs > 0 else None,
            "autotune": {q: tune[q] for q in ("cta_slots_primal", "cta_slots_dual", "list_fraction",
                                              "list_warps_per_sm") if q in tune}}


def run_warm_start(args, dev, stream):
    """Learned warm start on the transportation family (300 sources x 300 sinks, 20,000 side
    rows: shared A, perturbed b and c): solve training instances with the plain solver,
    train the network on those solutions with the library's own kernels, then solve
    held-out instances from zero and from the network's prediction, guarded per instance
    (``gnn.guard_starts``: a prediction is kept only where its KKT error after 64 iterations
    is no worse than the cold start's).  Solves run batched (every instance with its own
    restarts and status).  The warm time includes inference and the guard's probes; power
    iteration and graph capture are outside both timings."""
    import numpy as np
    import torch

    import lpgen
    from paper_2601_07628_gb300 import gnn
    from paper_2601_07628_gb300.dpdlp import Solver

    fam = lpgen.transport_family(seed=4)
    if args.x3_full:
        ntrain, ntest, epochs = 2000, 200, 8
    else:
        ntrain, ntest, epochs = args.ws_train, args.ws_test, args.ws_epochs
    tol_train, chunk = 1e-4, 200

    def solve(lps, tol, starts=None, guard=False):
        s = Solver(dev)
        s.set_stream(stream)
        s.load_batch(lps)
        s.solve(tol, 64)  # power iteration and graph capture, untimed
        s.set_param("resume", 0)
        t0 = time.perf_counter()
        keep = None
        if starts is not None:
            if guard:
                starts, keep, _, _ = gnn.guard_starts(s, lps, starts)
            else:
                s.set_start(np.concatenate([x for x, _ in starts]), np.concatenate([y for _, y in starts]))
        st = s.solve(tol, 2_000_000)
        dt = time.perf_counter() - t0
        x, y = s.solution()
        its = [k["iterations"] for k in s.batch_kkt()]
        parts = s.split(x, y)
        s.close()
        return st, dt, parts, its, keep

    t0 = time.perf_counter()
    train = [lpgen.transport_lp(fam, 100 + i) for i in range(ntrain)]
    test = [lpgen.transport_lp(fam, 1_000_000 + i) for i in range(ntest)]
    xs, ys, data_s = [], [], 0.0
    for a in range(0, ntrain, chunk):
        st, dt, parts, _, _ = solve(train[a:a + chunk], tol_train)
        data_s += dt
        xs += [x.copy() for x, _ in parts]
        ys += [y.copy() for _, y in parts]
    gen_s = time.perf_counter() - t0
    sc = gnn.fit_scales(train, xs, ys)
    net = gnn.Network(dev)
    net.set_params(gnn.init_params(0))
    net.set_graph(train[0].n, train[0].m, train[0].row_ptr, train[0].col, train[0].val)
    net.device_arrays(True)
    data = []
    for lp, x, y in zip(train, xs, ys):
        fv, fc = gnn.features(lp, sc)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(f"cuda:{dev}")
        data.append((t(fv), t(fc), t(x / sc.x_scale), t(y / sc.y_scale)))
    del xs, ys
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = gnn.train(net, data, epochs=epochs, lr=2e-3)
    train_s = time.perf_counter() - t0
    steps = epochs * ntrain
    del data
    t0 = time.perf_counter()
    starts = [gnn.predict(net, lp, sc) for lp in test]
    infer_s = time.perf_counter() - t0
    net.close()
    out = {"family": f"transportation {fam['S']} x {fam['D']} arcs + {fam['side'].shape[0]} side rows "
                     f"(n={train[0].n:,}, m={train[0].m:,}, nnz={train[0].nnz:,}), costs and "
                     f"supplies/demands perturbed per instance",
           "train_instances": ntrain, "train_tol": tol_train, "solve_train_s": data_s,
           "generate_and_solve_s": gen_s, "epochs": epochs, "train_s": train_s,
           "train_ms_per_step": 1e3 * train_s / steps, "loss_first_last": [hist[0], hist[-1]],
           "test_instances": ntest, "inference_s": infer_s,
           "guard": "a prediction is kept where its KKT error after 64 iterations is no worse "
                    "than the cold start's; the probes are inside the warm time"}
    for tol in (1e-6, 1e-8):
        stc, tc, _, itc, _ = solve(test, tol)
        stw, tw, _, itw, keep = solve(test, tol, starts, guard=True)
        out[f"{tol:.0e}"] = {
            "cold": {"status": stc, "seconds": tc, "median_iterations": float(np.median(itc)),
                     "mean_iterations": float(np.mean(itc)), "max_iterations": int(max(itc))},
            "warm": {"status": stw, "seconds": tw + infer_s, "median_iterations": float(np.median(itw)),
                     "mean_iterations": float(np.mean(itw)), "max_iterations": int(max(itw)),
                     "predictions_kept": int(sum(keep))},
            "instances_faster_warm": int(sum(w < c for w, c in zip(itw, itc))),
            "per_instance_iterations": {"cold": [int(v) for v in itc], "warm": [int(v) for v in itw]},
        }
    return out


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import numpy as np
    import torch

    from paper_2601_07628_gb300 import build
    from paper_2601_07628_gb300.costmodel import kernel_bytes
    from paper_2601_07628_gb300.dpdlp import Solver

    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
    build()
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream().cuda_stream
    dev = torch.cuda.current_device()
    if args.gnn_only:
        if rank == 0:
            run_gnn_only(args, dev)
        return

    lp = make_lp(args.workload)
    s = Solver(dev)
    s.set_stream(stream)
    s.load(lp)
    info = s.info()
    s.set_param("resume", 1)
    if args.host_loop:
        s.set_param("use_graph", 0)
    T = K_CHECK
    s.solve(0.0, T)  # power iteration and graph capture
    from paper_2601_07628_gb300 import autotune

    tuned = autotune.tune(s, cache=os.path.join(tempfile.gettempdir(), "dpdlp_autotune.json"),
                          reps=20, rounds=2, force=True)
    for _ in range(max(args.warmup, 3)):
        T += K_CHECK
        s.solve(0.0, T)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        T += K_CHECK
        s.solve(0.0, T)
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    value = job_throughput(args.steps * K_CHECK, world, ms)

    # ---- dominant kernel: average launch time with CUDA events on the solver's stream
    kb = kernel_bytes(lp.n, lp.m, lp.nnz)
    kt = {k: s.time_kernel(k, 50) for k in ("primal", "dual")}
    dom = max(kt, key=kt.get)
    peak, peak_kind = peaks()
    ach = kb[dom] / (kt[dom] * 1e-3) / 1e9
    # FP64 issue slots per launch: one FMA per nonzero plus the per-column / per-row updates
    fp64_ops = {"primal": lp.nnz + 8 * lp.n, "dual": lp.nnz + 9 * lp.m}
    sm_mhz = clk.get("sm_mhz") or 2070.0
    fp64_peak = N_SM * FP64_FMA_PER_CLK_SM * sm_mhz * 1e6 / 1e9  # G ops / s
    traffic = recorded_traffic(dom)
    roofline = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": traffic, "kernel": dom, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6800 GB/s",
                "bytes_per_launch": kb[dom], "ms_per_launch": kt[dom]}
    # (launches timed back to back as the solve runs them: programmatic dependents, each
    # launch's prologue overlapping the previous one's tail)
    kernels = {k: {"ms": kt[k], "GB/s": kb[k] / (kt[k] * 1e-3) / 1e9,
                   "hbm_frac": kb[k] / (kt[k] * 1e-3) / 1e9 / peak,
                   "fp64_Gops": fp64_ops[k] / (kt[k] * 1e-3) / 1e9,
                   "fp64_frac": fp64_ops[k] / (kt[k] * 1e-3) / 1e9 / fp64_peak}
               for k in kt}
    # ---- access ceilings of the packed layout: each kernel's loads without its arithmetic
    # (gather: indices + random x[col] gathers; access: + values; stream: indices + values;
    # memory: access + the epilogue's row-vector loads and stores)
    stored = {"primal": info["nnz_padded_csc"], "dual": info["nnz_padded_csr"]}
    for k in kt:
        # the slot kernel alone (without the long-row pass), the part the probes mirror
        kernels[k]["ms_slots_only"] = s.time_kernel(f"{k}_slots", 50)
        pr = {mode: s.time_kernel(f"{mode}_{k}", 50)
              for mode in ("gather", "access", "stream", "memory")}
        kernels[k]["ceilings"] = {
            mode: {"ms": t, "stored_entries": stored[k],
                   "G_entries_per_s": stored[k] / (t * 1e-3) / 1e9,
                   "kernel_frac": t / kt[k], "slot_kernel_frac": t / kernels[k]["ms_slots_only"]}
            for mode, t in pr.items()}
        kernels[k]["ceilings"]["stream"]["GB/s"] = 12 * stored[k] / (pr["stream"] * 1e-3) / 1e9
        kernels[k]["ceilings"]["gather"]["L2_sectors_per_s"] = stored[k] / (pr["gather"] * 1e-3)
    roofline["access_ceiling"] = {
        "what": "the dominant kernel's own loads (index and value streams + one random 8-byte "
                "gather of a 32-byte L2 sector per stored entry) without arithmetic, CUDA events",
        "ms_per_launch": kernels[dom]["ceilings"]["access"]["ms"],
        "kernel_frac": kernels[dom]["ceilings"]["access"]["kernel_frac"],
        "gather_only_ms": kernels[dom]["ceilings"]["gather"]["ms"],
        "stream_only_ms": kernels[dom]["ceilings"]["stream"]["ms"],
        "with_row_vectors_ms": kernels[dom]["ceilings"]["memory"]["ms"],
        "with_row_vectors_kernel_frac": kernels[dom]["ceilings"]["memory"]["kernel_frac"],
        "slot_kernel_ms": kernels[dom]["ms_slots_only"],
        "with_row_vectors_slot_kernel_frac": kernels[dom]["ceilings"]["memory"]["slot_kernel_frac"]}

    # ---- library reference point: cuSPARSE CSR SpMV (through torch) on the same matrix,
    # A x and A^T y in FP64, timed like the fused kernels (which do more: the product plus
    # the primal or dual step).  Not on the solver's path.
    spmv_ref = None
    try:
        spmv_ref = cusparse_reference(lp, dev, kb)
    except Exception as exc:  # report, do not fail the benchmark
        spmv_ref = {"error": str(exc)[:200]}

    # ---- the same steps without programmatic dependent launch between the iteration kernels
    s.set_param("pdl", 0)
    for k in kt:  # launch times without the overlap of consecutive launches
        kernels[k]["ms_without_pdl"] = s.time_kernel(k, 50)
    Tp = T
    for _ in range(2):
        Tp += K_CHECK
        s.solve(0.0, Tp)
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nq = max(args.steps // 2, 3)
    q0.record()
    for _ in range(nq):
        Tp += K_CHECK
        s.solve(0.0, Tp)
    q1.record()
    torch.cuda.synchronize()
    value_nopdl = job_throughput(nq * K_CHECK, world, max_over_ranks(q0.elapsed_time(q1), world))
    s.set_param("pdl", 1)

    # ---- mixed-precision form: FP32 matrix values (FP64 products), same steps
    s.set_param("spmv_fp32", 2)
    s.set_param("resume", 0)
    T32 = K_CHECK
    s.solve(0.0, T32)
    s.set_param("resume", 1)
    for _ in range(2):
        T32 += K_CHECK
        s.solve(0.0, T32)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n32 = max(args.steps // 2, 3)
    f0.record()
    for _ in range(n32):
        T32 += K_CHECK
        s.solve(0.0, T32)
    f1.record()
    torch.cuda.synchronize()
    value32 = job_throughput(n32 * K_CHECK, world, max_over_ranks(f0.elapsed_time(f1), world))
    kb32 = kernel_bytes(lp.n, lp.m, lp.nnz, val_bytes=4)
    kt32 = {k: s.time_kernel(k, 50) for k in ("primal", "dual")}
    forms = {"fp64": {"value": value, "unit": "iter/s"},
             "fp64_without_pdl": {"value": value_nopdl, "unit": "iter/s"},
             "fp32_values": {"value": value32, "unit": "iter/s",
                             "kernels": {k: {"ms": kt32[k], "GB/s": kb32[k] / (kt32[k] * 1e-3) / 1e9,
                                             "hbm_frac": kb32[k] / (kt32[k] * 1e-3) / 1e9 / peak}
                                         for k in kt32}}}
    s.set_param("spmv_fp32", 0)

    # ---- end to end through the C ABI with pinned host buffers
    xh = torch.empty(lp.n, dtype=torch.float64, pin_memory=True).numpy()
    yh = torch.empty(lp.m, dtype=torch.float64, pin_memory=True).numpy()
    xs, ys = s.solution()
    xh[:], yh[:] = xs, ys
    s.set_param("resume", 0)
    s.set_start(xh, yh)
    s.solve(0.0, K_CHECK)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.e2e_steps):
        s.set_start(xh, yh)
        s.solve(0.0, K_CHECK)
        s.solution(xh, yh)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
    e2e = {"value": job_throughput(args.e2e_steps * K_CHECK, world, e2e_ms), "unit": "iter/s",
           "h2d_bytes_per_step": 8 * (lp.n + lp.m), "d2h_bytes_per_step": 8 * (lp.n + lp.m),
           "step": "set_start(host x,y) + 64 iterations from it + get_solution(host)"}

    # ---- time to tolerance (plain FP64 and mixed precision)
    ttt = {}
    if args.tol_runs != "none" and rank == 0:
        if args.workload == "powerlaw" and args.tol_runs != "small":
            for mode in (0, 1):
                key = f"powerlaw_1e-4_{['fp64', 'mixed_fp32'][mode]}"
                ttt[key] = time_to_tol(s, 1e-4, 400_000, mode)
            if args.tol_runs == "all":
                ttt["powerlaw_1e-8_fp64"] = time_to_tol(s, 1e-8, 2_000_000, 0)
            # the same LP with the optional diagonal preconditioning (loaded again: the
            # scaling is a load-time step, reported in preprocess_ms)
            sp_ = Solver(dev)
            sp_.set_stream(stream)
            sp_.set_param("precond", 1)
            sp_.load(lp)
            runs = [(1e-4, 0), (1e-6, 0), (1e-8, 0)] + ([(1e-8, 1)] if args.tol_runs == "all" else [])
            for tol, mode in runs:
                r = time_to_tol(sp_, tol, 2_000_000, mode)
                r["preprocess_ms"] = sp_.info()["preprocess_ms"]
                ttt[f"powerlaw_{tol:.0e}_precond_{['fp64', 'mixed_fp32'][mode]}"] = r
            sp_.close()
        import lpgen

        # diagonal QP: a LASSO instance (min 1/2 ||M x - d||^2 + lam ||x||_1 as a QP), 20,000 x
        # 10,000 M with 0.2 % nonzeros
        if args.tol_runs != "small":
            qlp, _ = lpgen.lasso_qp(11, rows=20_000, cols=10_000, density=0.002, lam=0.5)
            sq = Solver(dev)
            sq.set_stream(stream)
            sq.load(qlp)
            for tol in (1e-4, 1e-6):
                ttt[f"lasso_qp_{tol:.0e}_fp64"] = time_to_tol(sq, tol, 400_000, 0)
            sq.close()

        sm = Solver(dev)
        sm.set_stream(stream)
        slp = lpgen.small_random_lp(0)
        sm.load(slp)
        for tol in (1e-4, 1e-8):
            answers = []
            for mode in (0, 1):
                ttt[f"small_lp_{tol:.0e}_{['fp64', 'mixed_fp32'][mode]}"] = time_to_tol(sm, tol, 1_000_000, mode)
                answers.append(solution_and_objective(sm))
            ttt[f"small_lp_{tol:.0e}_mixed_fp32"]["error_vs_fp64"] = error_vs_fp64(answers[1], answers[0],
                                                                                   slp.p_star)
        sm.close()
        # a tiny LP (n=250, m=125, 2 warp slots per packed copy) takes the fused body (one
        # launch per 64 iterations); the same solve with separate primal / dual launches
        st_ = Solver(dev)
        st_.set_stream(stream)
        st_.load(lpgen.small_random_lp(7, n=250, m=125))
        for fused in (1, 0):
            st_.set_param("fused_body", fused)
            r = time_to_tol(st_, 1e-8, 1_000_000, 0)
            r["fused_body"] = st_.info()["fused_body"]
            r["us_per_iteration"] = 1e6 * r["seconds"] / max(r["iterations"], 1)
            ttt[f"tiny_lp_1e-08_fp64_{['separate_launches', 'fused_body'][fused]}"] = r
        st_.close()
    s.close()
    batch = None
    if rank == 0 and args.workload == "powerlaw" and not args.no_batch:
        batch = run_batch(args, dev, stream, peak)
    warm = None
    if rank == 0 and args.workload == "powerlaw" and not args.no_warm_start:
        warm = run_warm_start(args, dev, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_subprocess(args.workload, args.cpu_sample_iters)

    if rank != 0:
        return
    launches_per_step = launches_per_body(info, 1)
    line = {
        "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.workload),
                   "step": f"{K_CHECK} fused PDHG iterations + 1 KKT/restart/PID check (one CUDA-graph body)",
                   "l2": "inputs larger than L2 (matrix CSR+CSC ~1 GB)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "block_permute": 1, "tiles_csr": info["tiles_csr"], "tiles_csc": info["tiles_csc"],
                   "pdl": 1,
                   "cta_slots": {"primal": tuned["cta_slots_primal"], "dual": tuned["cta_slots_dual"]}},
        "clocks": clk, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
        "roofline": roofline, "kernels": kernels, "spmv_cusparse": spmv_ref, "forms": forms,
        "fp64_peak_Gops": fp64_peak, "time_to_tol": ttt, "preprocess_ms": info["preprocess_ms"],
        "cpu_baseline": cpu, "batch": batch, "warm_start": warm,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
