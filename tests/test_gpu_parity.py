"""GPU path vs the FP64 CPU oracle, through the C ABI (needs a GB300).

Parity bar: after a fixed iteration count T, ||x_gpu - x_oracle|| / ||x_oracle|| <= 1e-9
and the same for y, with the oracle's restart decisions replayed on the GPU
(``dpdlp_set_schedule``) so that a decision flipped by last-bit rounding cannot split the
trajectories; the free-running decisions are compared separately.  The oracle's inputs
never come from the GPU: eta is the oracle's own power-iteration value (or a value the
test fixes), and the schedule flows from the oracle to the GPU only.
"""
import math

import numpy as np
import pytest

import lpgen
from oracle import pdhg as O
from parity_util import KKT_ABS, assert_xy_parity, first_divergence

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="session")
def Solver():
    from paper_2601_07628_gb300 import build, dpdlp

    build()
    return dpdlp.Solver


ORACLE_KEYS = ("gamma", "halpern", "check_every", "restart", "beta_sufficient", "beta_necessary",
               "beta_artificial", "pid", "pid_kp", "pid_ki", "pid_kd", "eta", "omega0")


def run_pair(Solver, lp, T, params=None, eta=None, eps=0.0, forced=True, permute=1, solver=None):
    params = dict(params or {})
    o = O.OracleLP.from_lpgen(lp)
    if eta is None:
        eta = O.default_eta(o)
    params["eta"] = eta
    ores = O.solve(o, eps=eps, max_iter=T, params=params)
    s = solver or Solver()
    s.set_param("block_permute", permute)
    s.load(lp)
    for k, v in params.items():
        if k in ORACLE_KEYS and v is not None:
            s.set_param(k, v)
    if forced:
        s.set_schedule([r["restart"] for r in ores.trace])
    status = s.solve(eps, T)
    x, y = s.solution()
    return ores, s, status, x, y


def assert_parity(ores, x, y, tol=TOL):
    assert_xy_parity(x, y, ores.x, ores.y, tol)


# --------------------------------------------------------------------------- small LP
@pytest.mark.parametrize("T", [1, 2, 63, 64, 65, 200, 1000, 5000])
def test_small_lp_fixed_iterations(Solver, T):
    lp = lpgen.small_random_lp(0)
    ores, s, status, x, y = run_pair(Solver, lp, T)
    assert status == 1
    assert_parity(ores, x, y)
    k = s.kkt()
    assert k["iterations"] == T and k["restarts"] == ores.restarts
    for key in ("r_primal", "r_dual", "r_gap"):
        assert math.isclose(k[key], ores.kkt[key], rel_tol=1e-6, abs_tol=KKT_ABS), key
    assert abs(k["omega"] - ores.omega) <= 1e-9 * ores.omega


@pytest.mark.parametrize("permute", [0, 1])
@pytest.mark.parametrize("seed", [1, 2])
def test_free_running_schedule_matches(Solver, seed, permute):
    lp = lpgen.small_random_lp(seed, n=1500, m=700)
    ores, s, status, x, y = run_pair(Solver, lp, 640, forced=False, permute=permute)
    rep = first_divergence(s.trace(), ores.trace)  # the first differing decision, if any
    assert rep is None, rep
    assert_parity(ores, x, y)
    tr = s.trace()
    for a, b in zip(tr, ores.trace):
        assert a["T"] == b["T"]
        assert math.isclose(a["r_fp"], b["r"], rel_tol=1e-7)
        assert math.isclose(a["omega"], b["omega"], rel_tol=1e-9)


@pytest.mark.parametrize("variant", [dict(halpern=0), dict(gamma=0.5), dict(gamma=0.0),
                                     dict(restart=0), dict(pid=0), dict(check_every=17),
                                     dict(check_every=1)])
def test_variants(Solver, variant):
    lp = lpgen.small_random_lp(3, n=800, m=400, nnz_per_col=6)
    ores, s, status, x, y = run_pair(Solver, lp, 300, params=variant)
    assert_parity(ores, x, y)


def test_converges_to_1e4_and_1e8(Solver):
    lp = lpgen.small_random_lp(0)
    o = O.OracleLP.from_lpgen(lp)
    eta = O.default_eta(o)
    for eps in (1e-4, 1e-8):
        ores = O.solve(o, eps=eps, max_iter=200000, params=dict(eta=eta))
        s = Solver()
        s.load(lp)
        s.set_param("eta", eta)
        status = s.solve(eps, 200000)
        assert status == 0 and ores.status == 0
        k = s.kkt()
        assert max(k["r_primal"], k["r_dual"], k["r_gap"]) <= eps
        assert abs(k["iterations"] - ores.iterations) <= 4 * 64
        assert abs(k["obj_p"] - lp.p_star) / (1 + abs(lp.p_star)) <= 50 * eps


# --------------------------------------------------------------------------- tile shapes
# Row lengths around every boundary of the lane packing: rows that fill a lane exactly (32),
# rows one longer (a full piece plus a one-nonzero tail), multiples of 32, long rows of many
# pieces, empty rows, and runs of one-nonzero rows that hit the per-slot row budget.
STRESS_LENGTHS = ([0, 1, 7, 8, 9, 31, 32, 33, 0, 0, 255, 256, 257, 511, 512, 513, 1000, 1023,
                   1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097, 8191, 8192, 8193, 9000, 0]
                  + [5] * 600 + [0, 3000, 16385, 30000] + [17] * 200 + [1] * 900 + [0, 0])


@pytest.fixture(scope="module")
def stress_lp():
    return lpgen.row_length_stress_lp(11, STRESS_LENGTHS, n=40000)


def test_spmv_tiles_against_oracle(Solver, stress_lp):
    """A x and A^T y on rows/columns of every tile kind (empty rows, rows straddling
    thread and tile boundaries, single-chunk and multi-chunk long rows)."""
    lp = stress_lp
    o = O.OracleLP.from_lpgen(lp)
    s = Solver()
    s.load(lp)
    rng = np.random.default_rng(0)
    for _ in range(3):
        x = rng.standard_normal(lp.n)
        y = rng.standard_normal(lp.m)
        ax, aty = s.apply_A(x), s.apply_AT(y)
        np.testing.assert_allclose(ax, o.Ax(x), rtol=1e-12, atol=1e-12 * np.abs(x).max() * 100)
        np.testing.assert_allclose(aty, o.ATy(y), rtol=1e-12, atol=1e-12 * np.abs(y).max() * 100)
    info = s.info()
    assert info["long_rows"] >= 3 and info["nnz"] == lp.nnz


def test_stress_lp_iterations(Solver, stress_lp):
    ores, s, status, x, y = run_pair(Solver, stress_lp, 130)
    assert_parity(ores, x, y)


@pytest.mark.parametrize("per_col", [3000, 10000])
def test_long_columns(Solver, per_col):
    """Few columns with thousands of nonzeros: the CSC pass splits them into lane pieces
    that the long-row pass adds in order."""
    lp = lpgen.small_random_lp(4, n=40, m=12000, nnz_per_col=per_col)
    ores, s, status, x, y = run_pair(Solver, lp, 100)
    assert_parity(ores, x, y)
    assert s.info()["long_cols"] == lp.n


def test_general_bounds(Solver):
    """Ranged, '>=', free rows and free / one-sided variables (set_row_bounds path)."""
    lp = lpgen.small_random_lp(5, n=900, m=450, nnz_per_col=5)
    rng = np.random.default_rng(1)
    lc, uc = lp.lc.copy(), lp.uc.copy()
    kind = rng.integers(0, 4, lp.m)
    ax = O.OracleLP.from_lpgen(lp).Ax(lp.x_star)
    lc = np.where(kind == 0, ax - 0.5, np.where(kind == 1, ax - 0.3, np.where(kind == 2, -np.inf, lc)))
    uc = np.where(kind == 0, ax + 0.5, np.where(kind == 1, np.inf, np.where(kind == 2, np.inf, uc)))
    lv, uv = lp.lv.copy(), lp.uv.copy()
    fv = rng.random(lp.n) < 0.1
    lv[fv] = -np.inf
    uv[fv] = np.inf
    g = lpgen.LP(lp.n, lp.m, lp.c, lp.row_ptr, lp.col, lp.val, lc, uc, lv, uv, name="general")
    ores, s, status, x, y = run_pair(Solver, g, 256)
    assert_parity(ores, x, y)


def test_box_only_and_empty_columns(Solver):
    rng = np.random.default_rng(2)
    n = 50
    c = rng.standard_normal(n)
    lp = lpgen.LP(n, 0, c, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), np.zeros(0),
                  np.zeros(0), -np.ones(n), np.ones(n), name="box")
    ores, s, status, x, y = run_pair(Solver, lp, 100, eta=1.0)
    assert_parity(ores, x, y)
    s2 = Solver()
    s2.load(lp)
    assert s2.solve(1e-10, 100000) == 0
    np.testing.assert_allclose(s2.solution()[0], np.where(c > 0, -1.0, 1.0), atol=1e-9)


# --------------------------------------------------------------------------- determinism, state
def test_bitwise_deterministic_and_graph_equals_host_loop(Solver):
    lp = lpgen.small_random_lp(6, n=1200, m=600)
    outs = []
    for use_graph in (1, 1, 0):
        s = Solver()
        s.set_param("use_graph", use_graph)
        s.load(lp)
        s.set_param("eta", 0.1)
        s.solve(0.0, 500)
        outs.append(s.solution())
    for x, y in outs[1:]:
        assert np.array_equal(x, outs[0][0]) and np.array_equal(y, outs[0][1])


def test_fresh_solve_on_a_used_handle_is_a_new_handle(Solver):
    """A fresh solve depends on nothing an earlier solve on the same handle left behind
    (iterates, scalars, the built graph), and a start point set earlier is used until it
    is cleared: after set_start() the solve is bitwise that of a new handle."""
    lp = lpgen.small_random_lp(7, n=1000, m=500)
    new = Solver()
    new.load(lp)
    new.solve(1e-6, 640)
    ref = new.solution(), new.kkt()["iterations"]
    used = Solver()
    used.load(lp)
    used.solve(1e-6, 64)
    used.set_start(np.ones(lp.n), np.ones(lp.m))
    used.solve(1e-6, 640)
    warm1 = used.solution()
    used.solve(1e-6, 640)  # the start is still set: the same warm solve again
    warm2 = used.solution()
    assert np.array_equal(warm1[0], warm2[0]) and np.array_equal(warm1[1], warm2[1])
    assert not np.array_equal(warm1[0], ref[0][0])  # it did start elsewhere
    used.set_start()
    used.solve(1e-6, 640)
    got = used.solution()
    assert np.array_equal(got[0], ref[0][0]) and np.array_equal(got[1], ref[0][1])
    assert used.kkt()["iterations"] == ref[1]
    new.close()
    used.close()


def test_schedule_replacement_frees_the_old_buffer(Solver):
    """Each dpdlp_set_schedule replaces the device buffer of the previous schedule: the
    handle's device memory stays the same over many calls, and the last schedule is the
    one in force."""
    lp = lpgen.small_random_lp(3, n=200, m=100)
    s = Solver()
    s.load(lp)
    s.set_schedule([0, 3, 0])
    before = s.info()["device_bytes"]
    for _ in range(50):
        s.set_schedule([0, 3, 0])
    assert s.info()["device_bytes"] == before
    s.set_schedule([3, 0, 0, 3])
    s.solve(0.0, 4 * 64)
    assert [r["restart"] for r in s.trace()] == [3, 0, 0, 3]
    s.close()


def test_checkpoint_resume_is_exact(Solver):
    lp = lpgen.small_random_lp(7, n=1000, m=500)
    a = Solver()
    a.load(lp)
    a.set_param("eta", 0.1)
    a.solve(0.0, 384)
    full = a.solution()
    b = Solver()
    b.load(lp)
    b.set_param("eta", 0.1)
    b.solve(0.0, 192)
    st = b.get_state()
    c = Solver()
    c.load(lp)
    c.set_state(st)
    c.solve(0.0, 384)
    got = c.solution()
    assert np.array_equal(got[0], full[0]) and np.array_equal(got[1], full[1])
    assert c.kkt()["restarts"] == a.kkt()["restarts"]


def test_planted_optimum_is_a_fixed_point(Solver):
    lp = lpgen.small_random_lp(8, n=600, m=300)
    s = Solver()
    s.load(lp)
    s.set_start(lp.x_star, lp.y_star)
    s.solve(0.0, 200)
    x, y = s.solution()
    np.testing.assert_allclose(x, lp.x_star, atol=1e-11)
    np.testing.assert_allclose(y, lp.y_star, atol=1e-11)


def test_warm_start_parity(Solver):
    lp = lpgen.small_random_lp(9, n=700, m=350)
    rng = np.random.default_rng(3)
    x0 = lp.x_star + 0.1 * rng.standard_normal(lp.n)
    y0 = lp.y_star + 0.1 * rng.standard_normal(lp.m)
    o = O.OracleLP.from_lpgen(lp)
    ores = O.solve(o, eps=0.0, max_iter=150, params=dict(eta=0.1), x_start=x0, y_start=y0)
    s = Solver()
    s.load(lp)
    s.set_param("eta", 0.1)
    s.set_schedule([r["restart"] for r in ores.trace])
    s.set_start(x0, y0)
    s.solve(0.0, 150)
    x, y = s.solution()
    assert_parity(ores, x, y)


def test_time_kernel_keeps_state(Solver):
    lp = lpgen.small_random_lp(10, n=1000, m=500)
    s = Solver()
    s.load(lp)
    s.set_param("eta", 0.1)
    s.solve(0.0, 64)
    before = s.get_state()
    assert s.time_kernel("primal", 5) > 0 and s.time_kernel("dual", 5) > 0
    assert s.time_kernel("primal_slots", 5) > 0 and s.time_kernel("dual_slots", 5) > 0
    # the access probes, including the one that stores into the epilogue's output vectors
    for probe in ("gather", "access", "stream", "memory"):
        for side in ("primal", "dual"):
            assert s.time_kernel(f"{probe}_{side}", 3) > 0
    after = s.get_state()
    for k in ("x", "y", "x0", "y0"):
        assert np.array_equal(before[k], after[k])
    # and the solve continues exactly as one that was never timed
    s.solve(0.0, 128)
    t = Solver()
    t.load(lp)
    t.set_param("eta", 0.1)
    t.solve(0.0, 64)
    t.solve(0.0, 128)
    for a, b in zip(s.solution(), t.solution()):
        assert np.array_equal(a, b)


def test_invalid_inputs_are_rejected(Solver):
    from paper_2601_07628_gb300.dpdlp import DpdlpError

    lp = lpgen.small_random_lp(0, n=20, m=10, nnz_per_col=2)
    s = Solver()
    with pytest.raises(DpdlpError) as e:
        s.solve(1e-4, 10)
    assert e.value.code == -4
    bad = lpgen.LP(**{**lp.__dict__})
    bad.col = lp.col.copy()
    bad.col[0] = lp.n
    with pytest.raises(DpdlpError) as e:
        s.load(bad)
    assert e.value.code == -1
    bad = lpgen.LP(**{**lp.__dict__})
    bad.lv = lp.lv.copy()
    bad.lv[0] = 100.0
    bad.uv = lp.uv.copy()
    bad.uv[0] = 1.0
    with pytest.raises(DpdlpError):
        s.load(bad)
    bad = lpgen.LP(**{**lp.__dict__})
    bad.val = lp.val.copy()
    bad.val[3] = np.nan
    with pytest.raises(DpdlpError):
        s.load(bad)
    novar = lpgen.LP(0, 3, np.zeros(0), np.zeros(4, np.int64), np.zeros(0, np.int32), np.zeros(0),
                     np.zeros(3), np.zeros(3), np.zeros(0), np.zeros(0), name="no variables")
    with pytest.raises(DpdlpError) as e:  # an LP needs a variable: rejected before any upload
        s.load(novar)
    assert e.value.code == -1
    with pytest.raises(DpdlpError) as e:  # so does each instance of a batch
        s.load_batch([lp, novar])
    assert e.value.code == -1
    with pytest.raises(DpdlpError):
        s.set_param("no_such_key", 1.0)
    with pytest.raises(DpdlpError):
        s.set_param("check_every", 0)


# --------------------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def big_lp():
    return lpgen.powerlaw_lp(1)


def test_powerlaw_full_size_parity(Solver, big_lp):
    """The 4M x 2M, 40M-nonzero power-law LP in the benchmark's launch configuration
    (graph loop, check every 64, block permutation on): whole-vector parity after 2 and
    after 64 iterations (one check with restart logic).  eta = 1/||A||_F (a valid step,
    since ||A||_2 <= ||A||_F), fixed by the test."""
    lp = big_lp
    eta = 1.0 / float(np.linalg.norm(lp.val))
    for T in (2, 64):
        ores, s, status, x, y = run_pair(Solver, lp, T, eta=eta)
        assert_parity(ores, x, y)
        k = s.kkt()
        for key in ("r_primal", "r_dual", "r_gap"):
            assert math.isclose(k[key], ores.kkt[key], rel_tol=1e-6), key
        s.close()
