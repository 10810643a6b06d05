"""Pins of the oracle's optional diagonal preconditioning (oracle/precond.py), on the CPU.

Pinned by: the power-of-two rounding rule on exact values; exactness of the scaled LP;
equilibration of a badly scaled matrix; invariance of the reported KKT errors under the
scaling (the primal residual and both objectives are those of the original LP at the
mapped point); the identity case reproducing the plain solve bit for bit; and convergence
to the planted optimum of a generator LP at 1e-8.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
from oracle import pdhg as O
from oracle import precond as P


def test_pow2_nearest():
    v = np.array([1.0, 8.0, 2 ** -10, 1.41 * 4, 1.42 * 4, 0.75, 0.7, 3.0, 5.0, 2 ** 0.5 * 0.999])
    want = np.array([1.0, 8.0, 2 ** -10, 4.0, 8.0, 1.0, 0.5, 4.0, 4.0, 1.0])
    assert np.array_equal(P.pow2_nearest(v), want)
    # the geometric midpoint 2^(k + 1/2) is the boundary
    for k in (-3, 0, 5):
        assert P.pow2_nearest(2.0 ** (k + 0.5) * (1 + 1e-12)) == 2.0 ** (k + 1)
        assert P.pow2_nearest(2.0 ** (k + 0.5) * (1 - 1e-12)) == 2.0 ** k


def badly_scaled(seed=0, m=60, n=90):
    rng = np.random.default_rng(seed)
    A = sp.random(m, n, density=0.1, random_state=np.random.RandomState(seed),
                  data_rvs=lambda k: rng.uniform(0.5, 2.0, k) * rng.choice([-1, 1], k)).tocsr()
    A = (sp.diags(10.0 ** rng.uniform(-6, 6, m)) @ A @ sp.diags(10.0 ** rng.uniform(-6, 6, n))).tocsr()
    A.sort_indices()
    return A


def test_factors_are_powers_of_two_and_scaling_is_exact():
    A = badly_scaled()
    lp = O.OracleLP(A.shape[1], A.shape[0], np.ones(A.shape[1]), A.indptr, A.indices, A.data,
                    -np.ones(A.shape[0]), np.ones(A.shape[0]), np.zeros(A.shape[1]),
                    np.full(A.shape[1], 3.0))
    dr, dc = P.scale_factors(lp)
    for d in (dr, dc):
        mant, _ = np.frexp(d)
        assert np.all(mant == 0.5)
    S = P.scaled_lp(lp, dr, dc)
    r, c = A.nonzero()
    Sd = S.A.toarray()
    assert np.array_equal(Sd[r, c], A.toarray()[r, c] * dr[r] * dc[c])
    x = np.random.default_rng(1).standard_normal(A.shape[1])
    assert np.array_equal((x / dc) * dc, x)  # conversions are exact


def test_ruiz_equilibrates():
    A = badly_scaled(3)
    lp = O.OracleLP(A.shape[1], A.shape[0], np.ones(A.shape[1]), A.indptr, A.indices, A.data,
                    -np.ones(A.shape[0]), np.ones(A.shape[0]), np.zeros(A.shape[1]),
                    np.ones(A.shape[1]))
    dr, dc = P.scale_factors(lp, ruiz_passes=30, pock_chambolle=False)
    S = abs(P.scaled_lp(lp, dr, dc).A)
    rmax = S.max(axis=1).toarray().ravel()
    cmax = S.max(axis=0).toarray().ravel()
    rmax, cmax = rmax[rmax > 0], cmax[cmax > 0]
    before = abs(A).max(axis=1).toarray().ravel()
    assert before.max() / before[before > 0].min() > 1e6
    assert rmax.max() <= 4.0 and rmax.min() >= 0.25
    assert cmax.max() <= 4.0 and cmax.min() >= 0.25


def test_kkt_is_reported_for_the_original_lp():
    lp = lpgen.small_random_lp(2, n=300, m=150)
    o = O.OracleLP.from_lpgen(lp)
    dr, dc = P.scale_factors(o)
    S = P.scaled_lp(o, dr, dc)
    rng = np.random.default_rng(5)
    x = np.clip(rng.standard_normal(o.n), o.lv, o.uv)
    y = rng.standard_normal(o.m)
    y[~np.isfinite(o.lc)] = -np.abs(y[~np.isfinite(o.lc)])  # a dual point in Y: p(-y) finite
    bn, cn = O.finite_bound_norm(o.lc, o.uc), float(np.linalg.norm(o.c))
    ks = O.kkt(S, x / dc, y / dr, 0.3, bn, cn, 1.0 / dr, 1.0 / dc)
    ko = O.kkt(o, x, y, 0.3)
    assert ks["r_primal"] == pytest.approx(ko["r_primal"], rel=1e-12)
    assert ks["obj_p"] == pytest.approx(ko["obj_p"], rel=1e-12)
    # with D_c = I the projected dual step is the same step, so every value agrees
    S1 = P.scaled_lp(o, dr, np.ones(o.n))
    k1 = O.kkt(S1, x, y / dr, 0.3, bn, cn, 1.0 / dr, np.ones(o.n))
    for key in ("r_primal", "r_dual", "r_gap", "obj_p", "obj_d"):
        assert k1[key] == pytest.approx(ko[key], rel=1e-12, abs=1e-14), key


def test_identity_scaling_is_the_plain_solve():
    lp = lpgen.small_random_lp(0)
    o = O.OracleLP.from_lpgen(lp)
    a = O.solve(o, eps=0.0, max_iter=200)
    b = P.solve(o, eps=0.0, max_iter=200, ruiz_passes=0, pock_chambolle=False)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y)
    assert a.kkt == b.kkt


def test_preconditioned_solve_reaches_planted_optimum():
    lp = lpgen.small_random_lp(1)
    o = O.OracleLP.from_lpgen(lp)
    res = P.solve(o, eps=1e-8, max_iter=200_000)
    assert res.status == 0
    assert max(res.kkt["r_primal"], res.kkt["r_dual"], res.kkt["r_gap"]) <= 1e-8
    assert abs(float(lp.c @ res.x) - lp.p_star) <= 1e-6 * (1 + abs(lp.p_star))
    # independent check in the original variables
    ax = o.Ax(res.x)
    assert np.linalg.norm(ax - O.proj_S(ax, o.lc, o.uc)) <= 1e-6 * (1 + np.linalg.norm(lp.b))
    assert np.all(res.x >= o.lv - 1e-12) and np.all(res.x <= o.uv + 1e-12)


def test_preconditioned_answer_satisfies_the_original_kkt():
    """The pair returned by the preconditioned solve, mapped back (x = D_c xs, y = D_r ys), is
    optimal for the original LP: its KKT errors evaluated on the original LP, with nothing
    of the scaling, are at the solve's tolerance (an optimal pair has zero projected-gradient
    residual for every step size, so the step size of this check is free)."""
    lp = lpgen.small_random_lp(1)
    o = O.OracleLP.from_lpgen(lp)
    res = P.solve(o, eps=1e-8, max_iter=200_000)
    assert res.status == 0
    for tau in (0.1, 1.0):
        k = O.kkt(o, res.x, res.y, tau)
        assert max(k["r_primal"], k["r_dual"], k["r_gap"]) <= 1e-7, (tau, k)
    # the reported primal residual and primal objective are the original LP's: the factors
    # are powers of two, so the scaled residual divided by D_r is the original one exactly
    dr, dc = P.scale_factors(o)
    assert not np.all(dr == 1.0)  # the check below would not see inverted row weights
    assert res.kkt["r_primal"] == pytest.approx(k["r_primal"], rel=1e-12)
    assert res.kkt["obj_p"] == pytest.approx(k["obj_p"], rel=1e-12)
