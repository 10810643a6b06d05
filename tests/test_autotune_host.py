"""Host logic of the launch-shape autotuner (no GPU): size classes, the choice rule and the
JSON cache, driven by a stand-in solver that records what is applied."""
import json

from paper_2601_07628_gb300 import autotune


class FakeSolver:
    """Stand-in for dpdlp.Solver: launch times come from tables, a large single LP never
    fits the fused body; batches answer the list and idle timings."""

    def __init__(self, times, n=4000, m=2000, nnz=40000, ninst=1, batch_times=None):
        self.times = times  # {(kernel, w): ms}
        self.batch_times = batch_times or {}  # {suffix: ms} or {("_list", warps): ms}
        self.params = {"cta_slots_primal": 4, "cta_slots_dual": 4, "spmv_fp32": 0,
                       "fused_body": 1, "fused_max_slots": 6, "list_fraction": 0.5,
                       "list_warps_per_sm": 0}
        self.row_off = list(range(ninst + 1))
        self._info = dict(n=n, m=m, nnz=nnz, fused_body=0, tiles_csr=40, tiles_csc=40)
        self.timed = 0

    def info(self):
        return dict(self._info)

    def get_param(self, k):
        return self.params[k]

    def set_param(self, k, v):
        self.params[k] = v

    def time_kernel(self, kern, reps):
        self.timed += 1
        side, _, suffix = kern.partition("_")
        if not suffix:
            return self.times[(kern, self.params[autotune.PARAMS[kern]])]
        key = ("_list", self.params["list_warps_per_sm"]) if suffix == "list" else "_" + suffix
        return self.batch_times[key] / 2  # the primal and the dual launch each half


def test_crossover_rule():
    # list walk: 10 % dearer per active slot, nearly free when idle; launch over every slot:
    # its idle cost is a fifth of the full launch.  Lines 0.2 + 0.8 f and 0.01 + 1.09 f.
    f = autotune.crossover(a=1.0, l=1.1, e=0.2, c=0.01)
    assert abs(f - (0.2 - 0.01) / (1.09 - 0.8)) < 1e-12
    assert autotune.crossover(1.0, 0.9, 0.2, 0.01) == 2.0  # list never dearer: always
    assert autotune.crossover(1.0, 0.9, 0.01, 0.2) == 0.0  # list dearer when idle: never
    assert abs(autotune.crossover(1.0, 5.0, 0.2, 0.19) - 0.01 / 4.01) < 1e-15


def test_tune_batch_sets_list_parameters(tmp_path):
    times = {(k, w): 1.0 for k in ("primal", "dual") for w in autotune.VARIANTS}
    bt = {("_list", 8): 1.3, ("_list", 16): 1.1, ("_list", 24): 1.2, "_idle": 0.2,
          "_list_idle": 0.01}
    s = FakeSolver(times, ninst=8, batch_times=bt)
    r = autotune.tune(s, cache=str(tmp_path / "c.json"), reps=1, rounds=1)
    assert r["list_warps_per_sm"] == 16 and s.params["list_warps_per_sm"] == 16
    want = autotune.crossover(2.0, 1.1, 0.2, 0.01)
    assert abs(r["list_fraction"] - want) < 1e-12 and s.params["list_fraction"] == r["list_fraction"]
    s2 = FakeSolver(times, ninst=8, batch_times=bt)
    r2 = autotune.tune(s2, cache=str(tmp_path / "c.json"))
    assert r2["cached"] and s2.timed == 0 and s2.params["list_warps_per_sm"] == 16


def test_size_class_buckets():
    a = autotune.size_class(dict(n=4_000_000, m=2_000_000, nnz=39_963_981), 1, False, "dev")
    b = autotune.size_class(dict(n=3_000_000, m=1_500_000, nnz=34_000_000), 1, False, "dev")
    c = autotune.size_class(dict(n=4_000_000, m=2_000_000, nnz=39_963_981), 256, False, "dev")
    d = autotune.size_class(dict(n=4_000_000, m=2_000_000, nnz=39_963_981), 1, True, "dev")
    assert a == b and len({a, c, d}) == 3
    assert a == "dev/n22_m21_z26_b0_fp64"


def test_choose_fastest_and_ties():
    assert autotune.choose({2: 1.0, 4: 0.9, 8: 0.95}) == 4
    assert autotune.choose({2: 1.0, 4: 1.0, 8: 1.0}) == 2


def test_tune_applies_and_caches(tmp_path):
    path = str(tmp_path / "cache.json")
    times = {("primal", 2): 0.30, ("primal", 4): 0.20, ("primal", 8): 0.25,
             ("dual", 2): 0.18, ("dual", 4): 0.19, ("dual", 8): 0.22}
    s = FakeSolver(times)
    r = autotune.tune(s, cache=path, reps=5, rounds=2)
    assert not r["cached"] and r["cta_slots_primal"] == 4 and r["cta_slots_dual"] == 2
    assert s.params["cta_slots_primal"] == 4 and s.params["cta_slots_dual"] == 2
    data = json.load(open(path))
    assert data[r["key"]]["cta_slots_dual"] == 2
    # a second handle of the same class takes the cached choice without timing
    s2 = FakeSolver({k: 1.0 for k in times})
    r2 = autotune.tune(s2, cache=path)
    assert r2["cached"] and s2.timed == 0 and s2.params["cta_slots_dual"] == 2
    # force re-times and overwrites
    r3 = autotune.tune(s2, cache=path, force=True)
    assert not r3["cached"] and r3["cta_slots_dual"] == 2 and s2.timed > 0


def test_corrupt_cache_is_ignored(tmp_path):
    path = tmp_path / "cache.json"
    path.write_text("{not json")
    times = {(k, w): float(w) for k in ("primal", "dual") for w in autotune.VARIANTS}
    r = autotune.tune(FakeSolver(times), cache=str(path), reps=1, rounds=1)
    assert r["cta_slots_primal"] == 2 and json.load(open(path))[r["key"]]["cta_slots_primal"] == 2
