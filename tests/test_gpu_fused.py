"""The fused body for small LPs (parameters ``fused_body``, ``fused_max_slots``,
``fused_cluster``): all iterations of a graph body in one launch of one thread block, or
of one thread-block cluster whose CTAs share the slots and exchange x_bar and y through
distributed shared memory.

Both forms run the same lane sums, epilogues and long-row sums as the separate primal and
dual launches, in the same order, so every result must be bitwise equal to the separate
path (compared as raw 64-bit patterns), and at parity with the oracle like the separate path.
The tests force the fused form (``fused_max_slots`` = 64) on LPs larger than the default
threshold, so that many slots per warp and long rows are covered: the cross-stress LP has
long rows in both orientations (rows of A with 1,500 and 1,100 nonzeros, a column with
1,200).
"""
import dataclasses

import numpy as np
import pytest

import lpgen
from oracle import pdhg as O
from parity_util import assert_xy_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def Solver():
    from paper_2601_07628_gb300 import build, dpdlp

    build()
    return dpdlp.Solver


def cross_lp():
    return lpgen.cross_stress_lp(5, [1500, 1100, 200, 40, 0, 1, 33] + [12] * 1493, 2000,
                                 {5: 1200, 7: 600, 9: 40})


def small_qp():
    lp = lpgen.small_random_lp(0)
    rng = np.random.default_rng(50)
    q = np.where(rng.random(lp.n) < 0.5, rng.uniform(0.1, 2.0, lp.n), 0.0)
    return dataclasses.replace(lp, q=q, x_star=None)


def run(Solver, lp, fused, T, eps=0.0, **params):
    s = Solver()
    s.set_param("fused_body", fused)
    s.set_param("fused_max_slots", 64)
    for k, v in params.items():
        s.set_param(k, v)
    s.load(lp)
    st = s.solve(eps, T)
    x, y = s.solution()
    out = dict(status=st, x=x, y=y, kkt=s.kkt(), info=s.info(), trace=s.trace())
    s.close()
    return out


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.int64)


CASES = {
    "small": (lpgen.small_random_lp, {}),
    "cross": (cross_lp, {}),
    "qp": (small_qp, {}),
    "fp32_values": (lpgen.small_random_lp, dict(spmv_fp32=2)),
    "host_loop": (cross_lp, dict(use_graph=0)),
    "check_every_17": (cross_lp, dict(check_every=17)),
    "no_halpern": (lpgen.small_random_lp, dict(halpern=0)),
}


@pytest.mark.parametrize("cluster", [1, 3, 8])
@pytest.mark.parametrize("case", list(CASES))
def test_fused_body_is_bitwise_the_separate_path(Solver, case, cluster):
    make, params = CASES[case]
    lp = make()
    T = 333  # not a multiple of the check period: the last body stops early
    a = run(Solver, lp, 1, T, fused_cluster=cluster, **params)
    b = run(Solver, lp, 0, T, **params)
    assert a["info"]["fused_body"] == 1 and b["info"]["fused_body"] == 0
    assert a["status"] == b["status"] == 1
    assert np.array_equal(bits(a["x"]), bits(b["x"]))
    assert np.array_equal(bits(a["y"]), bits(b["y"]))
    for key in ("iterations", "restarts", "checks", "r_primal", "r_dual", "r_gap", "omega"):
        assert a["kkt"][key] == b["kkt"][key], key
    assert [r["restart"] for r in a["trace"]] == [r["restart"] for r in b["trace"]]


@pytest.mark.parametrize("cluster", [1, 2, 8])
@pytest.mark.parametrize("case", ["tiny", "small", "cross", "fp32_values"])
def test_slot_cache_is_bitwise_the_uncached_body(Solver, case, cluster):
    """Each block's copy of its slots in shared memory (``fused_slot_cache``, on by default
    where it fits) changes where the product reads the matrix, not what it adds: bitwise the
    same results as reading the global slots."""
    lp = {"tiny": lambda: lpgen.small_random_lp(3, n=250, m=125), "small": lpgen.small_random_lp,
          "cross": cross_lp, "fp32_values": lpgen.small_random_lp}[case]()
    params = dict(spmv_fp32=2) if case == "fp32_values" else {}
    a = run(Solver, lp, 1, 333, fused_cluster=cluster, fused_slot_cache=1, **params)
    b = run(Solver, lp, 1, 333, fused_cluster=cluster, fused_slot_cache=0, **params)
    assert a["info"]["fused_body"] == 1 and a["status"] == b["status"]
    assert np.array_equal(bits(a["x"]), bits(b["x"]))
    assert np.array_equal(bits(a["y"]), bits(b["y"]))
    for key in ("iterations", "restarts", "checks", "r_primal", "r_dual", "r_gap", "omega"):
        assert a["kkt"][key] == b["kkt"][key], key


def test_fused_body_long_rows_present(Solver):
    info = run(Solver, cross_lp(), 1, 1)["info"]
    assert info["long_rows"] >= 2 and info["long_cols"] >= 1
    assert info["tiles_csr"] <= 64 and info["tiles_csc"] <= 64


def test_fused_body_matches_oracle(Solver):
    lp = cross_lp()
    o = O.OracleLP.from_lpgen(lp)
    eta = O.default_eta(o)
    T = 300
    res = O.solve(o, eps=0.0, max_iter=T, params=dict(eta=eta))
    s = Solver()
    s.set_param("fused_max_slots", 64)
    s.load(lp)
    assert s.info()["fused_body"] == 1
    s.set_param("eta", eta)
    s.set_schedule([r["restart"] for r in res.trace])
    s.solve(0.0, T)
    x, y = s.solution()
    s.close()
    assert_xy_parity(x, y, res.x, res.y, 1e-9)


def test_fused_body_solves_to_1e8(Solver):
    lp = lpgen.small_random_lp(0)
    a = run(Solver, lp, 1, 200_000, eps=1e-8)
    b = run(Solver, lp, 0, 200_000, eps=1e-8)
    assert a["status"] == 0 and b["status"] == 0
    assert a["kkt"]["iterations"] == b["kkt"]["iterations"]
    assert max(a["kkt"][k] for k in ("r_primal", "r_dual", "r_gap")) <= 1e-8
    assert np.array_equal(bits(a["x"]), bits(b["x"]))


def test_large_lp_does_not_fuse(Solver):
    lp = lpgen.small_random_lp(1, n=20000, m=10000)
    info = run(Solver, lp, 1, 1)["info"]
    assert info["fused_body"] == 0


def test_default_threshold(Solver):
    """By default LPs with at most 48 slots per packed copy (``fused_max_slots``) take the
    fused form (one block up to 6 slots, a cluster beyond); larger ones launch separately."""
    tiny = lpgen.small_random_lp(7, n=250, m=125)  # 2 slots per copy
    small = lpgen.small_random_lp(0)  # 16 slots per copy
    big = lpgen.small_random_lp(1, n=8000, m=4000)  # 64 slots per copy
    for lp, want in ((tiny, 1), (small, 1), (big, 0)):
        s = Solver()
        s.load(lp)
        assert s.info()["fused_body"] == want
        s.close()
    a = run(Solver, tiny, 1, 500)
    b = run(Solver, tiny, 0, 500)
    assert np.array_equal(bits(a["x"]), bits(b["x"])) and np.array_equal(bits(a["y"]), bits(b["y"]))


def test_autotune_times_the_fused_body_and_keeps_the_state(Solver, tmp_path):
    """For a tiny single LP the autotuner times one graph body fused and separate from a
    saved state and restores it: the solver state is the same before and after."""
    from paper_2601_07628_gb300 import autotune

    lp = lpgen.small_random_lp(7, n=250, m=125)
    s = Solver()
    s.load(lp)
    s.solve(0.0, 64)
    before = s.get_state()
    r = autotune.tune(s, cache=str(tmp_path / "t.json"), reps=3, rounds=1)
    after = s.get_state()
    assert 1 <= r["fused_max_slots"] <= 64 and s.get_param("fused_max_slots") == r["fused_max_slots"]
    assert r["ms"]["body"]["fused"] > 0 and r["ms"]["body"]["separate"] > 0
    for k in ("x", "y", "x0", "y0"):
        assert np.array_equal(before[k], after[k]), k
    assert before["scalars"] == after["scalars"]
    s.close()
