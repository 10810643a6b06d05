"""Optional diagonal preconditioning on the GPU against the oracle (oracle/precond.py).

The GPU scales the LP on the host at load (power-of-two Ruiz and Pock-Chambolle factors),
iterates on the scaled LP and reports solutions and KKT errors of the original one; the
oracle does the same with its own code.  Same 1e-9 parity bar as the plain path.
"""

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


def oracle_run(lp, T, eps=0.0):
    o = O.OracleLP.from_lpgen(lp)
    dr, dc = P.scale_factors(o)
    eta = O.default_eta(P.scaled_lp(o, dr, dc))
    res = P.solve(o, eps=eps, max_iter=T, params=dict(eta=eta))
    return res, eta


@pytest.mark.parametrize("T", [64, 200, 1000])
def test_precond_matches_oracle(Solver, T):
    lp = lpgen.small_random_lp(0)
    res, eta = oracle_run(lp, T)
    s = Solver()
    s.set_param("precond", 1)
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


def test_precond_converges_to_1e8(Solver):
    lp = lpgen.small_random_lp(1)
    s = Solver()
    s.set_param("precond", 1)
    s.load(lp)
    assert s.solve(1e-8, 500_000) == 0
    k = s.kkt()
    assert max(k["r_primal"], k["r_dual"], k["r_gap"]) <= 1e-8
    x, _ = s.solution()
    assert abs(float(lp.c @ x) - lp.p_star) <= 1e-6 * (1 + abs(lp.p_star))
    s.close()


def test_precond_checkpoint_and_operator(Solver):
    lp = lpgen.small_random_lp(7, n=1000, m=500)
    a = Solver()
    a.set_param("precond", 1)
    a.load(lp)
    a.solve(0.0, 640)
    b = Solver()
    b.set_param("precond", 1)
    b.load(lp)
    b.solve(0.0, 320)
    st = b.get_state()
    c = Solver()
    c.set_param("precond", 1)
    c.load(lp)
    c.set_state(st)
    c.solve(0.0, 640)
    for u, v in zip(a.solution(), c.solution()):
        assert np.array_equal(u, v)
    # the operator at the boundary is the original A
    import scipy.sparse as sp

    A = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
    xv = np.random.default_rng(3).standard_normal(lp.n)
    yv = np.random.default_rng(4).standard_normal(lp.m)
    assert rel(a.apply_A(xv), A @ xv) <= 1e-13
    assert rel(a.apply_AT(yv), A.T @ yv) <= 1e-13
    for s in (a, b, c):
        s.close()


def test_precond_batch_equals_single_solves(Solver):
    lps = [lpgen.small_random_lp(0), lpgen.uneven_lp(101, 700), lpgen.uneven_lp(102, 2600)]
    s = Solver()
    s.set_param("precond", 1)
    s.load_batch(lps)
    assert s.solve(1e-6, 200_000) == 0
    x, y = s.solution()
    kk = s.batch_kkt()
    for i, (lp, (xi, yi)) in enumerate(zip(lps, s.split(x, y))):
        a = Solver()
        a.set_param("precond", 1)
        a.set_param("perm_seed", 1 + 2 * i)
        a.load(lp)
        assert a.solve(1e-6, 200_000) == 0
        xa, ya = a.solution()
        assert np.array_equal(xi, xa) and np.array_equal(yi, ya), i
        assert kk[i]["iterations"] == a.kkt()["iterations"]
        a.close()
    s.close()


def test_precond_full_size_two_iterations(Solver):
    """The 4M x 2M power-law LP, preconditioned, two iterations against the oracle (eta =
    0.998 / ||D_r A D_c||_F, fixed by the test)."""
    lp = lpgen.powerlaw_lp(1)
    o = O.OracleLP.from_lpgen(lp)
    dr, dc = P.scale_factors(o)
    S = P.scaled_lp(o, dr, dc)
    eta = 0.998 / float(np.linalg.norm(S.A.data))
    res = P.solve(o, eps=0.0, max_iter=2, params=dict(eta=eta))
    s = Solver()
    s.set_param("precond", 1)
    s.load(lp)
    s.set_param("eta", eta)
    s.solve(0.0, 2)
    x, y = s.solution()
    assert_xy_parity(x, y, res.x, res.y, 1e-9)
    s.close()
