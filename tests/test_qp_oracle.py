"""Pins of the oracle's diagonal-QP variant (Section "Extensions to Diagonal QPs"), CPU only.

The primal step becomes argmin over the box of 1/2 Q_jj x^2 + (c_j - (A^T y)_j) x +
(x - x_j)^2 / (2 tau), a clamped 1-D quadratic minimum.  Pinned by: q = 0 reproducing the
LP bit for bit; the prox step by hand; a separable box QP against its closed form; an
equality-constrained QP against its KKT linear system; a small QP with bounds and ranged
rows against an independent solver (scipy's SLSQP); and the KKT errors at those optima.
"""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.sparse as sp

import lpgen
from oracle import pdhg as O


def qp(A, c, lc, uc, lv, uv, q):
    A = sp.csr_matrix(A)
    A.sort_indices()
    return O.OracleLP(A.shape[1], A.shape[0], c, A.indptr, A.indices, A.data, lc, uc, lv, uv, q)


def test_zero_q_is_the_lp():
    lp = lpgen.small_random_lp(0)
    o = O.OracleLP.from_lpgen(lp)
    oq = O.OracleLP(lp.n, lp.m, lp.c, lp.row_ptr, lp.col, lp.val, lp.lc, lp.uc, lp.lv, lp.uv,
                    np.zeros(lp.n))
    a = O.solve(o, eps=0.0, max_iter=200)
    b = O.solve(oq, eps=0.0, max_iter=200)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y) and a.kkt == b.kkt


def test_prox_step_by_hand():
    # one variable, no rows: x = 1, c = 3, q = 2, tau = 0.5: (1 - 1.5) / (1 + 1) = -0.25
    o = qp(np.zeros((0, 1)), [3.0], [], [], [-np.inf], [np.inf], [2.0])
    xh, _, xbar, _ = O.pdhg_step(o, np.array([1.0]), np.zeros(0), 0.5, 1.0)
    assert xh[0] == -0.25 and xbar[0] == -1.5
    o2 = qp(np.zeros((0, 1)), [3.0], [], [], [0.0], [np.inf], [2.0])
    assert O.pdhg_step(o2, np.array([1.0]), np.zeros(0), 0.5, 1.0)[0][0] == 0.0


def test_separable_box_qp_closed_form():
    rng = np.random.default_rng(1)
    n = 50
    q = rng.uniform(0.5, 3.0, n)
    c = rng.normal(0, 3, n)
    lv, uv = -rng.uniform(0, 2, n), rng.uniform(0, 2, n)
    o = qp(np.zeros((0, n)), c, [], [], lv, uv, q)
    res = O.solve(o, eps=1e-12, max_iter=100_000, params=dict(eta=0.5))
    assert res.status == 0
    assert np.allclose(res.x, np.clip(-c / q, lv, uv), rtol=0, atol=1e-10)


def test_equality_qp_matches_kkt_system():
    rng = np.random.default_rng(2)
    n, m = 30, 12
    A = rng.normal(size=(m, n)) * (rng.random((m, n)) < 0.4)
    A[np.arange(m), np.arange(m)] += 1.0  # full row rank
    q = rng.uniform(0.5, 2.0, n)
    c = rng.normal(size=n)
    b = rng.normal(size=m)
    # stationarity Q x + c - A^T y = 0, feasibility A x = b
    K = np.block([[np.diag(q), -A.T], [A, np.zeros((m, m))]])
    sol = np.linalg.solve(K, np.concatenate([-c, b]))
    xs, ys = sol[:n], sol[n:]
    o = qp(A, c, b, b, np.full(n, -np.inf), np.full(n, np.inf), q)
    res = O.solve(o, eps=1e-10, max_iter=500_000)
    assert res.status == 0
    assert np.allclose(res.x, xs, atol=1e-7) and np.allclose(res.y, ys, atol=1e-7)
    k = O.kkt(o, xs, ys, 0.1)
    assert max(k["r_primal"], k["r_dual"], k["r_gap"]) < 1e-12


def test_bounded_qp_matches_slsqp():
    rng = np.random.default_rng(3)
    n, m = 8, 4
    A = rng.normal(size=(m, n))
    q = rng.uniform(0.2, 2.0, n)
    c = rng.normal(size=n)
    x0 = rng.uniform(0, 1, n)
    ax = A @ x0
    lc = ax - rng.uniform(0.1, 1.0, m)
    uc = ax + rng.uniform(0.1, 1.0, m)
    uc[0] = lc[0] = ax[0]  # one equality row
    lc[1] = -np.inf        # one '<=' row
    lv, uv = np.zeros(n), np.full(n, 2.0)
    uv[:2] = np.inf
    o = qp(A, c, lc, uc, lv, uv, q)
    res = O.solve(o, eps=1e-10, max_iter=500_000)
    assert res.status == 0
    f = lambda x: 0.5 * np.dot(q * x, x) + c @ x
    cons = [{"type": "eq", "fun": lambda x: A[0] @ x - lc[0]},
            {"type": "ineq", "fun": lambda x: uc[1:] - A[1:] @ x},
            {"type": "ineq", "fun": lambda x: A[2:] @ x - lc[2:]}]
    ref = so.minimize(f, x0, jac=lambda x: q * x + c, constraints=cons,
                      bounds=list(zip(lv, np.where(np.isfinite(uv), uv, None))), method="SLSQP",
                      options=dict(ftol=1e-14, maxiter=1000))
    assert ref.success
    assert f(res.x) == pytest.approx(ref.fun, rel=1e-7, abs=1e-9)
    assert np.allclose(res.x, ref.x, atol=1e-5)


def test_lasso_reformulation_matches_ista():
    """LASSO min 1/2 ||M x - d||^2 + lam ||x||_1 as the diagonal QP
    min 1/2 r^T r + lam 1^T t  s.t.  M x - r = d,  -t <= x <= t  (Q = I on r, 0 on x and t),
    against an independent proximal-gradient (ISTA) solve of the original problem."""
    import lpgen as G

    lp, meta = G.lasso_qp(5, rows=40, cols=25, density=0.3, lam=0.3)
    o = O.OracleLP(lp.n, lp.m, lp.c, lp.row_ptr, lp.col, lp.val, lp.lc, lp.uc, lp.lv, lp.uv, lp.q)
    res = O.solve(o, eps=1e-9, max_iter=2_000_000)
    assert res.status == 0
    M, d, lam = meta["M"].toarray(), meta["d"], meta["lam"]
    x = np.zeros(M.shape[1])
    L = np.linalg.norm(M, 2) ** 2
    for _ in range(200_000):
        z = x - M.T @ (M @ x - d) / L
        x = np.sign(z) * np.maximum(np.abs(z) - lam / L, 0.0)
    obj = lambda x: 0.5 * np.sum((M @ x - d) ** 2) + lam * np.abs(x).sum()
    xq = res.x[meta["x"]]
    assert obj(xq) == pytest.approx(obj(x), rel=1e-7)
    assert np.allclose(xq, x, atol=1e-5)
