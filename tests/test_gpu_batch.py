"""Batched solve: many independent LPs in one handle, iterating together in the same kernels
with per-instance step sizes, primal weights, restarts and statuses.

Each instance of a batch must behave as if it were solved alone: against the FP64 oracle
(per instance, with its own forced restart schedule) at the usual 1e-9 bound, and bit for
bit against a single-LP solve of the same instance (same block permutation seed), since
an instance's rows are packed, summed and reduced exactly as in a single solve.
"""
import numpy as np
import pytest

import lpgen
from oracle import pdhg as O
from parity_util import KKT_ABS, assert_vec_parity, assert_xy_parity

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="session")
def Solver():
    from paper_2601_07628_gb300 import build, dpdlp

    build()
    return dpdlp.Solver


def small_batch():
    """Uneven instances: the 2,000 x 1,000 LP, batch-workload instances of several sizes
    (one above the 4,096-element reduction chunk) and an LP whose rows and columns are
    longer than a lane (40 nonzeros per column, 100 per row)."""
    lps = [lpgen.small_random_lp(0)]
    lps += [lpgen.uneven_lp(100 + i, m) for i, m in enumerate((500, 777, 2600, 1300))]
    lps.append(lpgen.small_random_lp(4, n=300, m=120, nnz_per_col=40))
    return lps


@pytest.mark.parametrize("T", [64, 200, 1000])
def test_batch_matches_oracle_per_instance(Solver, T):
    lps = small_batch()
    etas, ores = [], []
    for lp in lps:
        o = O.OracleLP.from_lpgen(lp)
        eta = O.default_eta(o)
        etas.append(eta)
        ores.append(O.solve(o, eps=0.0, max_iter=T, params=dict(eta=eta)))
    s = Solver()
    s.load_batch(lps)
    s.set_batch_eta(etas)
    s.set_schedule([[r["restart"] for r in res.trace] for res in ores])
    assert s.solve(0.0, T) == 1
    x, y = s.solution()
    kk = s.batch_kkt()
    for i, ((xi, yi), res) in enumerate(zip(s.split(x, y), ores)):
        assert_xy_parity(xi, yi, res.x, res.y, TOL, f"instance {i}")
        assert kk[i]["restarts"] == res.restarts, i
        for key in ("r_primal", "r_dual", "r_gap"):
            assert kk[i][key] == pytest.approx(res.kkt[key], rel=1e-6, abs=KKT_ABS), (i, key)
    s.close()


def test_batch_instances_equal_single_solves(Solver):
    """Free-running restarts to 1e-6: every instance stops at its own check, with the same
    iterate, counters and residuals as the same LP solved alone."""
    lps = small_batch()
    s = Solver()
    s.load_batch(lps)
    assert s.solve(1e-6, 200_000) == 0
    x, y = s.solution()
    kk = s.batch_kkt()
    iters = set()
    for i, (lp, (xi, yi)) in enumerate(zip(lps, s.split(x, y))):
        a = Solver()
        a.set_param("perm_seed", 1 + 2 * i)
        a.load(lp)
        assert a.solve(1e-6, 200_000) == 0
        xa, ya = a.solution()
        ka = a.kkt()
        assert np.array_equal(xi, xa) and np.array_equal(yi, ya), i
        assert kk[i]["iterations"] == ka["iterations"] and kk[i]["restarts"] == ka["restarts"], i
        assert kk[i]["r_primal"] == ka["r_primal"] and kk[i]["omega"] == ka["omega"], i
        assert kk[i]["status"] == 0
        iters.add(ka["iterations"])
        a.close()
    assert len(iters) > 1  # the instances converge at different checks
    agg = s.kkt()
    assert agg["iterations"] == max(iters)
    assert agg["r_primal"] == max(k["r_primal"] for k in kk)
    s.close()


def test_batch_trace_and_statuses(Solver):
    lps = small_batch()[:3]
    s = Solver()
    s.load_batch(lps)
    s.solve(1e-6, 200_000)
    tr = s.trace()
    kk = s.batch_kkt()
    assert len(tr) % 3 == 0 and [r["inst"] for r in tr[:3]] == [0, 1, 2]
    last = tr[-3:]
    for i in range(3):
        assert last[i]["inst"] == i and last[i]["status"] == 0
        done = [r for r in tr if r["inst"] == i and r["status"] == 0]
        assert done[0]["T"] == kk[i]["iterations"]  # first record after its convergence
    s.close()


def test_batch_mixed_precision_per_instance(Solver):
    """Mixed precision in a batch: every instance switches to FP64 values on its own and
    reaches 1e-8."""
    lps = small_batch()[:4]
    s = Solver()
    s.set_param("spmv_fp32", 1)
    s.load_batch(lps)
    assert s.solve(1e-8, 500_000) == 0
    for k in s.batch_kkt():
        assert max(k["r_primal"], k["r_dual"], k["r_gap"]) <= 1e-8
        assert k["spmv_mode"] == 0
    s.close()


def test_batch_invalid_inputs(Solver):
    from paper_2601_07628_gb300 import dpdlp

    lps = small_batch()[:2]
    s = Solver()
    s.load_batch(lps)
    with pytest.raises(dpdlp.DpdlpError):
        s.set_schedule([1, 0, 0])  # not a multiple of the instance count
    with pytest.raises(dpdlp.DpdlpError):
        s.set_batch_eta([0.1])
    s.solve(0.0, 64)
    with pytest.raises(dpdlp.DpdlpError):
        s.get_state()  # checkpoints hold a single LP
    # a nonzero of instance 0's rows in instance 1's columns
    bad = [lpgen.small_random_lp(1, n=50, m=20), lpgen.small_random_lp(2, n=40, m=10)]
    bad[0].col[0] = 60
    with pytest.raises(dpdlp.DpdlpError):
        s.load_batch(bad)
    s.close()


def test_batch_with_empty_instance(Solver):
    """An instance without rows (a box-only LP) beside ordinary ones."""
    box = lpgen.small_random_lp(3, n=40, m=0)
    lps = [lpgen.uneven_lp(5, 600), box, lpgen.uneven_lp(6, 900)]
    etas, ores = [], []
    for lp in lps:
        o = O.OracleLP.from_lpgen(lp)
        etas.append(O.default_eta(o))
        ores.append(O.solve(o, eps=0.0, max_iter=300, params=dict(eta=etas[-1])))
    s = Solver()
    s.load_batch(lps)
    s.set_batch_eta(etas)
    s.set_schedule([[r["restart"] for r in res.trace] for res in ores])
    s.solve(0.0, 300)
    x, y = s.solution()
    for (xi, yi), res in zip(s.split(x, y), ores):
        assert_vec_parity(xi, res.x, TOL, "x")
        if yi.size:
            assert_vec_parity(yi, res.y, TOL, "y")
    s.close()


@pytest.fixture(scope="module")
def full_batch():
    return lpgen.batch_lps()


def test_full_batch_sampled_parity(Solver, full_batch):
    """The 256-LP batched workload (6.5M rows, 13.1M columns, 131M nonzeros) in the
    benchmark's launch configuration, 64 iterations (one check): the three smallest
    instances against the oracle.  One eta for all instances, 0.998 / max_i ||A_i||_F (a
    valid step for each, as ||A_i||_2 <= ||A_i||_F), fixed by the test."""
    lps = full_batch
    eta = 0.998 / max(float(np.linalg.norm(lp.val)) for lp in lps)
    s = Solver()
    s.load_batch(lps)
    s.set_param("eta", eta)
    T = 64
    assert s.solve(0.0, T) == 1
    x, y = s.solution()
    parts = s.split(x, y)
    kk = s.batch_kkt()
    for i in np.argsort([lp.m for lp in lps])[:3]:
        o = O.OracleLP.from_lpgen(lps[i])
        res = O.solve(o, eps=0.0, max_iter=T, params=dict(eta=eta))
        xi, yi = parts[i]
        assert_xy_parity(xi, yi, res.x, res.y, TOL, f"instance {i}")
        assert kk[i]["restarts"] == res.restarts
    s.close()


def test_launch_shapes_do_not_change_results(Solver):
    """Slots per block (2, 4, 8) of either iteration kernel, the list threshold (never /
    always walk the active-slot lists) and the list kernel's warps per SM are launch choices
    only: the batch solve gives bit-identical results under every combination."""
    lps = small_batch()
    ref = None
    for wp, wd, frac, lw in ((4, 4, 0.5, 0), (2, 2, 0.5, 0), (8, 8, 0.5, 0), (2, 8, 0.0, 0),
                             (8, 2, 2.0, 8), (4, 4, 2.0, 24), (4, 4, 0.9, 16)):
        s = Solver()
        s.set_param("cta_slots_primal", wp)
        s.set_param("cta_slots_dual", wd)
        s.set_param("list_fraction", frac)
        s.set_param("list_warps_per_sm", lw)
        s.load_batch(lps)
        assert s.solve(1e-6, 200_000) == 0
        x, y = s.solution()
        if ref is None:
            ref = (x, y)
        else:
            assert np.array_equal(x, ref[0]) and np.array_equal(y, ref[1]), (wp, wd, frac, lw)
        s.close()


def test_autotune_applies_and_caches(Solver, tmp_path):
    from paper_2601_07628_gb300 import autotune

    cache = str(tmp_path / "tune.json")
    s = Solver()
    s.load_batch(small_batch())
    r = autotune.tune(s, cache=cache, reps=5, rounds=1)
    assert not r["cached"]
    for p in autotune.PARAMS.values():
        assert r[p] in autotune.VARIANTS and s.get_param(p) == r[p]
    assert r["list_warps_per_sm"] in autotune.LIST_WARPS
    assert 0.0 <= r["list_fraction"] <= 2.0 and s.get_param("list_fraction") == r["list_fraction"]
    cr = r["ms"]["crossover"]
    assert all(v > 0 for v in cr.values()) and cr["list_idle"] < cr["all_running"]
    assert s.solve(1e-6, 200_000) == 0
    s2 = Solver()
    s2.load_batch(small_batch())
    r2 = autotune.tune(s2, cache=cache)
    assert r2["cached"] and r2["cta_slots_primal"] == r["cta_slots_primal"]
    s.close()
    s2.close()


def test_batch_graph_and_host_loop_agree(Solver):
    """The graph's device-side choice between the active-slot lists and one launch over every
    slot, and the host loop's choice of the same, give bit-identical results (the choice
    changes the launch, never the arithmetic)."""
    lps = small_batch()
    out = []
    for use_graph in (1, 0):
        s = Solver()
        s.set_param("use_graph", use_graph)
        s.load_batch(lps)
        assert s.solve(1e-6, 200_000) == 0
        out.append(s.solution())
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
