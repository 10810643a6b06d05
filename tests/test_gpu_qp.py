"""Diagonal QP on the GPU against the oracle (Section "Extensions to Diagonal QPs").

Same parity bar as the LP: 1e-9 after fixed iteration counts with the oracle's restart
decisions replayed; q = 0 must reproduce the LP bit for bit; the LASSO QP must reach the
LASSO optimum (cross-checked with an independent proximal-gradient solve).
"""
import dataclasses

import numpy as np
import pytest

import lpgen
from oracle import pdhg as O
from parity_util import KKT_ABS, assert_xy_parity, rel
from oracle import precond as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def Solver():
    from paper_2601_07628_gb300 import build, dpdlp

    build()
    return dpdlp.Solver


def oracle_lp(lp):
    return O.OracleLP(lp.n, lp.m, lp.c, lp.row_ptr, lp.col, lp.val, lp.lc, lp.uc, lp.lv, lp.uv,
                      lp.q)


def random_qp(seed=0):
    lp = lpgen.small_random_lp(seed)
    rng = np.random.default_rng(seed + 50)
    q = np.where(rng.random(lp.n) < 0.5, rng.uniform(0.1, 2.0, lp.n), 0.0)
    return dataclasses.replace(lp, q=q, x_star=None)


@pytest.mark.parametrize("case", ["lasso", "random"])
@pytest.mark.parametrize("T", [64, 500])
def test_qp_matches_oracle(Solver, case, T):
    lp = lpgen.lasso_qp(7, rows=300, cols=200, density=0.05, lam=0.2)[0] if case == "lasso" else random_qp()
    o = oracle_lp(lp)
    eta = O.default_eta(o)
    res = O.solve(o, eps=0.0, max_iter=T, params=dict(eta=eta))
    s = Solver()
    s.load(lp)
    s.set_param("eta", eta)
    s.set_schedule([r["restart"] for r in res.trace])
    s.solve(0.0, T)
    x, y = s.solution()
    assert_xy_parity(x, y, res.x, res.y, 1e-9)
    k = s.kkt()
    for key in ("r_primal", "r_dual", "r_gap", "obj_p", "obj_d"):
        assert k[key] == pytest.approx(res.kkt[key], rel=1e-6, abs=KKT_ABS), key
    s.close()


def test_zero_q_is_the_lp(Solver):
    lp = lpgen.small_random_lp(0)
    a = Solver()
    a.load(lp)
    a.solve(1e-6, 100_000)
    b = Solver()
    b.load(lp)
    b.set_objective_diag(np.zeros(lp.n))
    b.solve(1e-6, 100_000)
    for u, v in zip(a.solution(), b.solution()):
        assert np.array_equal(u, v)
    assert a.kkt()["iterations"] == b.kkt()["iterations"]
    a.close()
    b.close()


def test_lasso_reaches_its_optimum(Solver):
    lp, meta = lpgen.lasso_qp(8, rows=400, cols=250, density=0.05, lam=0.5)
    s = Solver()
    s.load(lp)
    assert s.solve(1e-8, 2_000_000) == 0
    x, _ = s.solution()
    k = s.kkt()
    assert max(k["r_primal"], k["r_dual"], k["r_gap"]) <= 1e-8
    M, d, lam = meta["M"].toarray(), meta["d"], meta["lam"]
    L = np.linalg.norm(M, 2) ** 2
    z = np.zeros(M.shape[1])
    for _ in range(100_000):
        w = z - M.T @ (M @ z - d) / L
        z = np.sign(w) * np.maximum(np.abs(w) - lam / L, 0.0)
    obj = lambda v: 0.5 * np.sum((M @ v - d) ** 2) + lam * np.abs(v).sum()
    assert obj(x[meta["x"]]) == pytest.approx(obj(z), rel=1e-6)
    s.close()


def test_preconditioned_qp_matches_oracle(Solver):
    lp = random_qp(1)
    o = oracle_lp(lp)
    dr, dc = P.scale_factors(o)
    eta = O.default_eta(P.scaled_lp(o, dr, dc))
    res = P.solve(o, eps=0.0, max_iter=200, params=dict(eta=eta))
    s = Solver()
    s.set_param("precond", 1)
    s.load(lp)
    s.set_param("eta", eta)
    s.set_schedule([r["restart"] for r in res.trace])
    s.solve(0.0, 200)
    x, y = s.solution()
    assert_xy_parity(x, y, res.x, res.y, 1e-9)
    s.close()


def test_batch_of_lps_and_qps(Solver):
    lps = [lpgen.small_random_lp(0), random_qp(2), lpgen.lasso_qp(9, rows=200, cols=120)[0]]
    s = Solver()
    s.load_batch(lps)
    assert s.solve(1e-6, 500_000) == 0
    x, y = s.solution()
    for i, (lp, (xi, yi)) in enumerate(zip(lps, s.split(x, y))):
        a = Solver()
        a.set_param("perm_seed", 1 + 2 * i)
        a.load(lp)
        assert a.solve(1e-6, 500_000) == 0
        xa, ya = a.solution()
        if lp.q is None:  # an LP instance of a batch with Q runs the QP kernel with q = 0
            assert rel(xi, xa) <= 1e-12 and rel(yi, ya) <= 1e-12, i
        else:
            assert np.array_equal(xi, xa) and np.array_equal(yi, ya), i
        a.close()
    s.close()
