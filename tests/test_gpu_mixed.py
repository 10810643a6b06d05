"""Mixed precision (FP32 matrix values, FP64 products and accumulation) vs the oracle.

With FP32 values the iteration is exactly FP64 PDHG on the LP whose matrix entries are
rounded to FP32 (a plain definition: ``val.astype(float32)``), so its iterates are compared
with the FP64 oracle run on that rounded LP at the usual 1e-9 bound.  The KKT checks keep
using the FP64 values, so reported residuals are those of the true LP; the mixed mode must
therefore switch to FP64 values to reach 1e-8.
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


def rounded(lp):
    return dataclasses.replace(lp, val=lp.val.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("T", [1, 64, 500])
def test_fp32_values_match_oracle_on_rounded_matrix(Solver, T):
    lp = lpgen.small_random_lp(0)
    lr = rounded(lp)
    o = O.OracleLP.from_lpgen(lr)
    eta = O.default_eta(o)
    ores = O.solve(o, eps=0.0, max_iter=T, params=dict(eta=eta))
    s = Solver()
    s.set_param("spmv_fp32", 2)
    s.load(lp)
    s.set_param("eta", eta)
    s.set_schedule([r["restart"] for r in ores.trace])
    s.solve(0.0, T)
    x, y = s.solution()
    assert_xy_parity(x, y, ores.x, ores.y, 1e-9)
    assert all(r["spmv_mode"] == 1 for r in s.trace())
    assert s.kkt()["spmv_mode"] == 1


def test_mixed_mode_switches_and_reaches_1e8(Solver):
    lp = lpgen.small_random_lp(0)
    s = Solver()
    s.set_param("spmv_fp32", 1)
    s.load(lp)
    assert s.solve(1e-8, 500000) == 0
    k = s.kkt()
    assert max(k["r_primal"], k["r_dual"], k["r_gap"]) <= 1e-8
    modes = [r["spmv_mode"] for r in s.trace()]
    assert modes[0] == 1 and modes[-1] == 0 and k["spmv_mode"] == 0
    assert abs(k["obj_p"] - lp.p_star) / (1 + abs(lp.p_star)) <= 1e-6


def test_mixed_mode_checkpoint_is_exact(Solver):
    lp = lpgen.small_random_lp(7, n=1000, m=500)
    a = Solver()
    a.set_param("spmv_fp32", 1)
    a.load(lp)
    a.set_param("eta", 0.1)
    a.solve(0.0, 640)
    b = Solver()
    b.set_param("spmv_fp32", 1)
    b.load(lp)
    b.set_param("eta", 0.1)
    b.solve(0.0, 320)
    st = b.get_state()
    c = Solver()
    c.load(lp)
    c.set_param("spmv_fp32", 1)
    c.set_state(st)
    c.solve(0.0, 640)
    for u, v in zip(a.solution(), c.solution()):
        assert np.array_equal(u, v)


def test_fp32_values_full_size(Solver):
    """Power-law LP, FP32 values, two iterations: whole-vector parity with the oracle on the
    rounded matrix (eta = 1/||A||_F fixed by the test)."""
    lp = lpgen.powerlaw_lp(1)
    lr = rounded(lp)
    eta = 1.0 / float(np.linalg.norm(lr.val))
    o = O.OracleLP.from_lpgen(lr)
    ores = O.solve(o, eps=0.0, max_iter=2, params=dict(eta=eta))
    s = Solver()
    s.set_param("spmv_fp32", 2)
    s.load(lp)
    s.set_param("eta", eta)
    s.solve(0.0, 2)
    x, y = s.solution()
    assert_xy_parity(x, y, ores.x, ores.y, 1e-9)
