"""Host logic of the launch-shape autotuner (no GPU): size classes, the choice rule and the
JSON cache, driven by a stand-in solver that records what is applied."""
import json

from paper_2601_07628_gb300 import autotune


class FakeSolver:
    def __init__(self, times, n=4000, m=2000, nnz=40000, ninst=1):
        self.times = times  # {(kernel, w): ms}
        self.params = {"cta_slots_primal": 4, "cta_slots_dual": 4, "spmv_fp32": 0}
        self.row_off = list(range(ninst + 1))
        self._info = dict(n=n, m=m, nnz=nnz)
        self.timed = 0

    def info(self):
        return dict(self._info)

    def get_param(self, k):
        return self.params[k]

    def set_param(self, k, v):
        self.params[k] = v

    def time_kernel(self, kern, reps):
        self.timed += 1
        return self.times[(kern, self.params[autotune.PARAMS[kern]])]


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
