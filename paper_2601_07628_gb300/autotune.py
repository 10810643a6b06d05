"""Launch autotuner for the iteration kernels, with a JSON cache per size class.

Every choice here changes how the work is launched, never the results:
* slots per thread block of the primal (A^T y) and dual (A x_bar) iteration kernels (2, 4
  or 8 warp slots: 64, 128 or 256 threads), timed per variant;
* batches: the resident warps per SM of the persistent kernel that walks the lists of
  slots of running instances (timed per variant), and the fraction of active slots below
  which a graph body walks those lists instead of launching over every slot.  The fraction
  is computed from four measured launch costs: a launch over every slot and the list walk
  with every instance running (a, l), and both with every instance stopped (e, c).  With a
  fraction f of the slots active a launch over every slot costs about e + f (a - e) and the
  list walk c + f (l - c); the crossover of the two lines is the threshold;
* a single LP small enough for the fused body: one graph body (check_every iterations and
  a check) timed fused and as separate launches from the same solver state, and
  fused_max_slots set so the faster form runs.
``tune`` uses the library's own event timer (``dpdlp_time_kernel``, which leaves the solver
state untouched) and, for the fused body, short solves between a saved and a restored
state.  It applies the choices and records them in a JSON cache keyed by the problem's size
class, so later handles of the same class skip the timing.

Size class: ceil(log2) of n, m, nnz and of the instance count, plus the value precision of
the products (FP64 or FP32 values) and the device name.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

VARIANTS = (2, 4, 8)
LIST_WARPS = (8, 16, 24)  # resident warps per SM of the persistent list kernel
PARAMS = {"primal": "cta_slots_primal", "dual": "cta_slots_dual"}
BATCH_PARAMS = ("list_fraction", "list_warps_per_sm")
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


def crossover(a: float, l: float, e: float, c: float) -> float:
    """Active-slot fraction below which the list walk is cheaper than a launch over every
    slot, for launch costs a, l (every instance running: over every slot, list walk) and
    e, c (every instance stopped).  The costs are taken as linear in the active fraction
    f: e + f (a - e) and c + f (l - c).  Returns a value in [0, 2]: 0 never walks the lists,
    2 always does."""
    slope_all, slope_list = a - e, l - c
    if slope_list <= slope_all:  # the list walk grows no faster: it wins from its crossing on
        return 2.0 if c <= e else 0.0
    f = (e - c) / (slope_list - slope_all)
    return float(min(2.0, max(0.0, f)))


def tune(solver, cache: str | None = DEFAULT_CACHE, reps: int = 20, rounds: int = 3,
         force: bool = False) -> dict:
    """Choose and apply the launch parameters for the loaded problem: the slots per block
    of both iteration kernels, and for a batch the list kernel's warps per SM and the
    list threshold, or for a single LP that fits the fused body, fused_max_slots.

    Needs a solver state (after ``solve`` or ``set_state``; a fresh handle gets one from a
    zero-iteration solve).  Returns ``{"key", "cached", "ms", <parameter>: <value>...}``;
    ``ms`` holds the timings (best of ``rounds`` x ``reps`` launches) when they were taken
    now.  Timing the fused body of a single LP runs graph bodies from a saved state and
    puts that state back with ``set_state``, so, as after any ``set_state``, the next
    ``solve`` continues from it whatever ``resume`` says.
    """
    info = solver.info()
    ninst = len(solver.row_off) - 1
    fp32 = bool(solver.get_param("spmv_fp32"))
    key = size_class(info, ninst, fp32)
    data = load_cache(cache) if cache else {}
    if not force and key in data:
        e = data[key]
        out = {"key": key, "cached": True, "ms": e.get("ms")}
        for p in list(PARAMS.values()) + list(BATCH_PARAMS) + ["fused_max_slots"]:
            if p in e:
                solver.set_param(p, e[p])
                out[p] = e[p]
        return out
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
    if ninst > 1:
        _tune_batch(solver, out, reps, rounds)
    else:
        _tune_fused(solver, out, rounds)
    if cache:
        data = load_cache(cache)
        data[key] = {k: v for k, v in out.items() if k not in ("key", "cached")}
        save_cache(cache, data)
    return out


def _pair(solver, suffix, reps, rounds):
    """Best-of-rounds time of the primal and dual launches of one kind, added."""
    tot = 0.0
    for kern in PARAMS:
        name = kern + suffix
        solver.time_kernel(name, reps)
        tot += min(solver.time_kernel(name, reps) for _ in range(rounds))
    return tot


def _tune_batch(solver, out, reps, rounds):
    times = {}
    for w in LIST_WARPS:
        solver.set_param("list_warps_per_sm", w)
        times[w] = _pair(solver, "_list", reps, rounds)
    best = choose(times)
    solver.set_param("list_warps_per_sm", best)
    a = _pair(solver, "", reps, rounds)
    l = times[best]
    e = _pair(solver, "_idle", reps, rounds)
    c = _pair(solver, "_list_idle", reps, rounds)
    f = crossover(a, l, e, c)
    solver.set_param("list_fraction", f)
    out["list_warps_per_sm"] = best
    out["list_fraction"] = f
    out["ms"]["list"] = {str(w): t for w, t in times.items()}
    out["ms"]["crossover"] = {"all_running": a, "list_running": l, "all_idle": e, "list_idle": c}


def _tune_fused(solver, out, rounds):
    """Time one graph body fused and separate from the same state (single LPs that fit)."""
    import time

    fused0, max0 = solver.get_param("fused_body"), solver.get_param("fused_max_slots")
    solver.set_param("fused_body", 1)
    solver.set_param("fused_max_slots", 64)
    fits = bool(solver.info()["fused_body"])
    solver.set_param("fused_body", fused0)
    solver.set_param("fused_max_slots", max0)
    if not fits:
        return
    state = solver.get_state()
    resume0 = solver.get_param("resume")
    K = int(solver.get_param("check_every"))
    T0 = int(state["scalars"]["T"])
    solver.set_param("resume", 1)
    t = {}
    for form in (1, 0):
        solver.set_param("fused_body", form)
        solver.set_param("fused_max_slots", 64)
        best = float("inf")
        for _ in range(rounds + 1):  # the first round builds the graph
            solver.set_state(state)
            t0 = time.perf_counter()
            solver.solve(0.0, T0 + 4 * K)
            best = min(best, time.perf_counter() - t0)
        t[form] = best / 4
    solver.set_state(state)
    solver.set_param("resume", resume0)
    solver.set_param("fused_body", fused0)
    info = solver.info()
    slots = max(info["tiles_csr"], info["tiles_csc"])
    mx = 64 if t[1] < t[0] else max(1, slots - 1)
    solver.set_param("fused_max_slots", mx)
    out["fused_max_slots"] = mx
    out["ms"]["body"] = {"fused": 1e3 * t[1], "separate": 1e3 * t[0]}
