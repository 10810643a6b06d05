"""Launch-shape autotuner for the iteration kernels, with a JSON cache per size class.

The primal (A^T y) and dual (A x_bar) iteration kernels process one warp slot per warp;
how many slots share a thread block (2, 4 or 8: 64, 128 or 256 threads) changes only the
launch shape, never the results.  ``tune`` times every variant of both kernels on the
loaded problem with the library's own event timer (``dpdlp_time_kernel``, which leaves the
solver state untouched), keeps the fastest, applies it, and records it in a JSON cache
keyed by the problem's size class, so later handles of the same class skip the timing.

Size class: ceil(log2) of n, m, nnz and of the instance count, plus the value precision of
the products (FP64 or FP32 values) and the device name.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

VARIANTS = (2, 4, 8)
PARAMS = {"primal": "cta_slots_primal", "dual": "cta_slots_dual"}
DEFAULT_CACHE = os.environ.get(
    "DPDLP_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "dpdlp", "autotune.json"))


def _lg(v: int) -> int:
    return int(math.ceil(math.log2(v))) if v > 1 else 0


def device_name() -> str:
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.get_device_name(0).replace(" ", "_")
    except Exception:
        pass
    return "cuda"


def size_class(info: dict, ninst: int, fp32: bool, device: str | None = None) -> str:
    return (f"{device or device_name()}/n{_lg(info['n'])}_m{_lg(info['m'])}_z{_lg(info['nnz'])}"
            f"_b{_lg(ninst)}_{'fp32' if fp32 else 'fp64'}")


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, data: dict) -> None:
    """Write atomically (temporary file + rename), so concurrent tuners never leave a torn file."""
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".autotune.", suffix=".json")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(times: dict) -> int:
    """Fastest variant; ties go to the smallest block (deterministic)."""
    return min(sorted(times), key=lambda w: (times[w], w))


def tune(solver, cache: str | None = DEFAULT_CACHE, reps: int = 20, rounds: int = 3,
         force: bool = False) -> dict:
    """Choose and apply the slots per block of both iteration kernels for the loaded problem.

    Needs a solver state (after ``solve`` or ``set_state``; a fresh handle gets one from a
    zero-iteration solve).  Returns ``{"key", "cta_slots_primal", "cta_slots_dual",
    "cached", "ms"}``; ``ms`` holds the timings (best of ``rounds`` x ``reps`` launches)
    when they were taken now.
    """
    info = solver.info()
    ninst = len(solver.row_off) - 1
    fp32 = bool(solver.get_param("spmv_fp32"))
    key = size_class(info, ninst, fp32)
    data = load_cache(cache) if cache else {}
    if not force and key in data:
        e = data[key]
        for k, p in PARAMS.items():
            solver.set_param(p, int(e[p]))
        return {"key": key, "cta_slots_primal": int(e["cta_slots_primal"]),
                "cta_slots_dual": int(e["cta_slots_dual"]), "cached": True, "ms": e.get("ms")}
    from .dpdlp import DpdlpError

    try:
        solver.time_kernel("primal", 1)
    except DpdlpError:  # no solver state yet: take one from a zero-iteration solve
        solver.solve(0.0, 0)
    out = {"key": key, "cached": False, "ms": {}}
    for kern, p in PARAMS.items():
        times = {}
        for w in VARIANTS:
            solver.set_param(p, w)
            solver.time_kernel(kern, reps)  # warm-up of this launch shape
            times[w] = min(solver.time_kernel(kern, reps) for _ in range(rounds))
        best = choose(times)
        solver.set_param(p, best)
        out[p] = best
        out["ms"][kern] = {str(w): t for w, t in times.items()}
    if cache:
        data = load_cache(cache)
        data[key] = {"cta_slots_primal": out["cta_slots_primal"],
                     "cta_slots_dual": out["cta_slots_dual"], "ms": out["ms"]}
        save_cache(cache, data)
    return out
