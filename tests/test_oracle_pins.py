"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each check ties one piece of the oracle to the paper or to mathematics: hand-computed
Chambolle-Pock iterates, closed-form optima, brute-force vertex enumeration, KKT values at
planted optima, a dense quadratic form for the P-norm, a library SVD for the power
iteration.  ``test_oracle_mutants.py`` plants plausible mistakes in the oracle and checks
that these pins catch each one.
"""
import itertools
import math

import numpy as np

import lpgen
import oracle
from oracle import pdhg as O

INF = np.inf


def one_var_lp(c=1.0):
    """min c x  s.t.  x >= 1 (one '>=' row),  0 <= x <= 5."""
    return O.OracleLP(1, 1, [c], [0, 1], [0], [1.0], [1.0], [INF], [0.0], [5.0])


# --------------------------------------------------------------------------- PDHG step
def check_pdhg_hand():
    """Section 2.2 with Halpern off is the textbook Chambolle-Pock step.  For
    min x s.t. x >= 1, 0 <= x <= 5 with tau = sigma = 1/2 from x = 0, y = 0, the textbook
    recursion x+ = clamp(x - tau(1 - y), 0, 5), y+ = max(0, y + sigma(1 - (2x+ - x))) gives,
    worked by hand:
      it1 (0, 1/2)   it2 (0, 1)   it3 (0, 3/2)   it4 (1/4, 7/4)   it5 (5/8, 7/4)
      it6 (1, 25/16)
    (all exact in binary64)."""
    lp = one_var_lp()
    expected = [(0.0, 0.5), (0.0, 1.0), (0.0, 1.5), (0.25, 1.75), (0.625, 1.75), (1.0, 1.5625)]
    x, y = np.zeros(1), np.zeros(1)
    for xe, ye in expected:
        xh, yh, _, _ = O.pdhg_step(lp, x, y, 0.5, 0.5)
        assert xh[0] == xe and yh[0] == ye, (xh, yh, xe, ye)
        x, y = xh, yh
    # the same through the full solve with Halpern and restarts off
    r = O.solve(lp, eps=0.0, max_iter=6, params=dict(eta=0.5, omega0=1.0, halpern=0, restart=0,
                                                      check_every=1000))
    assert r.x[0] == 1.0 and r.y[0] == 1.5625


def test_pdhg_step_hand_computed():
    check_pdhg_hand()


def check_dual_step_closed_forms():
    """The dual update of Section 2.2 equals, row by row, the prox of the conjugate:
    '=' row y+ = y + sigma (b - z); '<=' row min(0, .); '>=' row max(0, .); free row 0;
    ranged row [l, u]: y + sigma(l - z) if that is > 0, y + sigma(u - z) if that is < 0,
    else 0."""
    rng = np.random.default_rng(5)
    k = 400
    b = rng.standard_normal(k)
    for kind in ("eq", "le", "ge", "free", "ranged"):
        y = rng.standard_normal(k) * 2
        z = rng.standard_normal(k) * 2
        sigma = 0.37
        if kind == "eq":
            lc, uc = b, b
            want = y + sigma * (b - z)
        elif kind == "le":
            lc, uc = np.full(k, -INF), b
            want = np.minimum(0.0, y + sigma * (b - z))
        elif kind == "ge":
            lc, uc = b, np.full(k, INF)
            want = np.maximum(0.0, y + sigma * (b - z))
        elif kind == "free":
            lc, uc = np.full(k, -INF), np.full(k, INF)
            want = np.zeros(k)
        else:
            lc, uc = b - 0.5, b + 0.5
            lo = y + sigma * (lc - z)
            hi = y + sigma * (uc - z)
            want = np.where(lo > 0, lo, np.where(hi < 0, hi, 0.0))
        w = y / sigma - z
        got = sigma * (w - O.proj_negS(w, lc, uc))
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
        # the result lies in the dual set Y of Section 2.1 exactly
        if kind == "le":
            assert np.all(got <= 0.0)
        if kind == "ge":
            assert np.all(got >= 0.0)
        if kind == "free":
            assert np.all(got == 0.0)


def test_dual_step_closed_forms():
    check_dual_step_closed_forms()


# --------------------------------------------------------------------------- Halpern
def check_halpern_fixed_point():
    """Appendix B.1 with the affine reading: a fixed point z* of PDHG used as iterate and
    anchor stays put for every k and gamma (the weights sum to one)."""
    rng = np.random.default_rng(1)
    zs = rng.standard_normal(50)
    for k in (0, 1, 7, 100):
        for gamma in (0.0, 0.5, 1.0):
            out = O.halpern(zs, zs, zs, k, gamma)
            np.testing.assert_allclose(out, zs, rtol=1e-14, atol=1e-15)
    # k = 0, gamma = 1: z+ = (2T - z)/2 + z0/2 (hand value)
    t, z, z0 = np.array([3.0]), np.array([1.0]), np.array([-2.0])
    assert O.halpern(t, z, z0, 0, 1.0)[0] == (2 * 3.0 - 1.0) / 2 + (-2.0) / 2


def test_halpern_fixed_point_invariance():
    check_halpern_fixed_point()


def check_planted_optimum_is_fixed():
    """A saddle point is a fixed point of the whole restarted iteration: started at the
    planted (x*, y*) the oracle does not move (sign errors in either step would)."""
    lp = lpgen.small_random_lp(3, n=60, m=30, nnz_per_col=4)
    o = O.OracleLP.from_lpgen(lp)
    r = O.solve(o, eps=0.0, max_iter=130, params=dict(check_every=64), x_start=lp.x_star,
                y_start=lp.y_star)
    np.testing.assert_allclose(r.x, lp.x_star, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.y, lp.y_star, rtol=0, atol=1e-12)


def test_planted_optimum_is_fixed_point():
    check_planted_optimum_is_fixed()


# --------------------------------------------------------------------------- P-norm
def check_p_norm_dense():
    """Appendix D.2.1's expansion equals dz^T P dz with the dense metric P of Appendix B."""
    rng = np.random.default_rng(2)
    m, n = 5, 7
    A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.6)
    lp = lpgen.from_dense(A, np.zeros(n), np.zeros(m), np.zeros(m), np.zeros(n), np.ones(n))
    o = O.OracleLP.from_lpgen(lp)
    omega, eta = 1.7, 0.3
    Pm = np.block([[omega / eta * np.eye(n), A.T], [A, 1.0 / (eta * omega) * np.eye(m)]])
    for _ in range(5):
        dx, dy = rng.standard_normal(n), rng.standard_normal(m)
        dz = np.concatenate([dx, dy])
        want = dz @ Pm @ dz
        got = O.p_norm_sq(dx, dy, o.Ax(dx), omega, eta)
        assert abs(got - want) <= 1e-12 * max(1.0, abs(want))


def test_p_norm_matches_dense_metric():
    check_p_norm_dense()


# --------------------------------------------------------------------------- KKT
def check_kkt_hand():
    """Appendix B.4 formulas on min x, x >= 1, 0 <= x <= 5, worked by hand.

    At x = 1/2, y = 2, tau = 1/2: Ax = 1/2, proj_S = 1 -> r_p = (1/2)/(1+1) = 1/4;
    g = 1 - 2 = -1, x - tau g = 1, proj_X = 1 -> r_d = (1/2)/(1/2)/(1+1) = 1/2; s = 0;
    p(-y) = -l * 2 = -2 so obj_d = 2, obj_p = 1/2, r_gap = (3/2)/(1+2) = 1/2.

    For min -x at the optimum x = 5, y = 0, tau = 1/2: x - tau g = 11/2, proj_X = 5, s = -1,
    s^T x = -5 = obj_p, every residual 0."""
    k = O.kkt(one_var_lp(), np.array([0.5]), np.array([2.0]), 0.5)
    assert (k["r_primal"], k["r_dual"], k["r_gap"]) == (0.25, 0.5, 0.5)
    assert (k["obj_p"], k["obj_d"]) == (0.5, 2.0)
    k = O.kkt(one_var_lp(-1.0), np.array([5.0]), np.array([0.0]), 0.5)
    assert (k["r_primal"], k["r_dual"], k["r_gap"]) == (0.0, 0.0, 0.0)
    assert (k["obj_p"], k["obj_d"]) == (-5.0, -5.0)
    # min 3x with ||c|| = 3 != ||b|| = 1, at x = 1/2, y = 2, tau = 1/2: r_p = (1/2)/(1+1) = 1/4;
    # g = 3 - 2 = 1, x - tau g = 0 = proj_X -> r_d = (1/2)/(1/2)/(1+3) = 1/4, s = 0;
    # obj_p = 3/2, obj_d = 2, r_gap = (1/2)/(1+2)
    k = O.kkt(one_var_lp(3.0), np.array([0.5]), np.array([2.0]), 0.5)
    assert (k["r_primal"], k["r_dual"], k["r_gap"]) == (0.25, 0.25, 0.5 / 3.0)
    assert (k["obj_p"], k["obj_d"]) == (1.5, 2.0)


def test_kkt_hand_computed():
    check_kkt_hand()


def check_kkt_zero_at_planted():
    """At the generator's optimal pair every relative KKT error vanishes (to rounding) and
    both objectives equal p* = c^T x* (strong duality by construction)."""
    for seed in range(3):
        lp = lpgen.small_random_lp(seed, n=300, m=150, nnz_per_col=5)
        o = O.OracleLP.from_lpgen(lp)
        for tau in (0.01, 1.0):
            k = O.kkt(o, lp.x_star, lp.y_star, tau)
            assert max(k["r_primal"], k["r_dual"], k["r_gap"]) < 1e-13, k
            assert abs(k["obj_d"] - lp.p_star) <= 1e-11 * (1 + abs(lp.p_star))


def test_kkt_zero_at_planted_optimum():
    check_kkt_zero_at_planted()


def test_p_fun_zero_times_infinity():
    """p(y; l, u) = u^T y^+ - l^T y^- with 0 * inf = 0 (Section 2.1)."""
    y = np.array([2.0, -3.0, 0.0, 1.0])
    l = np.array([-INF, 1.0, -INF, 2.0])
    u = np.array([4.0, INF, INF, 5.0])
    assert O.p_fun(y, l, u) == 4.0 * 2.0 - 1.0 * 3.0 + 0.0 + 5.0 * 1.0


def test_finite_bound_norm():
    lc = np.array([1.0, -INF, 2.0, -1.0])
    uc = np.array([1.0, 3.0, INF, 4.0])
    assert O.finite_bound_norm(lc, uc) == math.sqrt(1 + 9 + 4 + 1 + 16)


# --------------------------------------------------------------------------- closed forms
def check_box_only():
    """With no rows the LP separates: x_j = l_j if c_j > 0 else u_j."""
    rng = np.random.default_rng(4)
    n = 9
    c = rng.standard_normal(n)
    l = -rng.uniform(0, 3, n)
    u = rng.uniform(0, 3, n)
    o = O.OracleLP(n, 0, c, [0], [], [], [], [], l, u)
    r = O.solve(o, eps=1e-10, max_iter=20000)
    assert r.status == 0
    np.testing.assert_allclose(r.x, np.where(c > 0, l, u), atol=1e-9)
    assert r.eta == 1.0 and r.y.shape == (0,)


def test_box_only_closed_form():
    check_box_only()


def check_knapsack():
    """Fractional knapsack max v^T x, w^T x <= W, 0 <= x <= 1: the greedy fill by v/w is
    optimal (one '<=' row exercises the sign-constrained dual)."""
    rng = np.random.default_rng(6)
    n = 12
    v = rng.uniform(1, 10, n)
    w = rng.uniform(1, 5, n)
    W = 0.4 * w.sum()
    order = np.argsort(-v / w)
    x = np.zeros(n)
    cap = W
    for j in order:
        take = min(1.0, cap / w[j])
        x[j] = take
        cap -= take * w[j]
        if cap <= 0:
            break
    best = float(v @ x)
    o = O.OracleLP(n, 1, -v, [0, n], np.arange(n), w, [-INF], [W], np.zeros(n), np.ones(n))
    r = O.solve(o, eps=1e-9, max_iter=200000)
    assert r.status == 0
    assert abs(-r.kkt["obj_p"] - best) <= 1e-7 * (1 + best)
    assert r.y[0] <= 0.0  # '<=' row: dual in R^-


def test_fractional_knapsack_closed_form():
    check_knapsack()


def brute_force_lp(lp):
    """Optimum of a bounded LP by enumerating every vertex: all n-subsets of constraint
    hyperplanes (rows and bounds, '=' rows as two), each solved by Gaussian elimination,
    feasible ones kept."""
    A = np.zeros((lp.m, lp.n))
    for i in range(lp.m):
        for e in range(lp.row_ptr[i], lp.row_ptr[i + 1]):
            A[i, lp.col[e]] = lp.val[e]
    G, h = [], []
    for i in range(lp.m):
        if np.isfinite(lp.uc[i]):
            G.append(A[i]); h.append(lp.uc[i])
        if np.isfinite(lp.lc[i]):
            G.append(-A[i]); h.append(-lp.lc[i])
    for j in range(lp.n):
        e = np.zeros(lp.n); e[j] = 1.0
        G.append(e); h.append(lp.uv[j])
        G.append(-e); h.append(-lp.lv[j])
    G, h = np.array(G), np.array(h)
    best = None
    for S in itertools.combinations(range(len(h)), lp.n):
        M = G[list(S)]
        if abs(np.linalg.det(M)) < 1e-10:
            continue
        x = np.linalg.solve(M, h[list(S)])
        if np.all(G @ x <= h + 1e-9):
            val = float(lp.c @ x)
            if best is None or val < best:
                best = val
    return best


def check_brute_force(seeds=range(6)):
    for seed in seeds:
        lp = lpgen.tiny_bounded_lp(seed, n=4, m=3)
        best = brute_force_lp(lp)
        o = O.OracleLP.from_lpgen(lp)
        r = O.solve(o, eps=1e-9, max_iter=400000)
        assert r.status == 0, (seed, r.kkt)
        assert abs(r.kkt["obj_p"] - best) / (1 + abs(best)) <= 1e-7, (seed, r.kkt, best)


def test_brute_force_vertex_enumeration():
    check_brute_force()


def check_generator_optimum(seeds=(0, 1)):
    """The oracle reaches the planted optimum p* of generator LPs at eps = 1e-8."""
    for seed in seeds:
        lp = lpgen.small_random_lp(seed, n=400, m=200, nnz_per_col=6)
        o = O.OracleLP.from_lpgen(lp)
        r = O.solve(o, eps=1e-8, max_iter=100000)
        assert r.status == 0
        err = abs(r.kkt["obj_p"] - lp.p_star) / (1 + abs(lp.p_star))
        assert err <= 1e-7, err


def test_generator_known_optimum():
    check_generator_optimum()


# --------------------------------------------------------------------------- step size
def check_power_iteration():
    """The power-iteration sigma_max matches the 2-norm from a library SVD."""
    rng = np.random.default_rng(7)
    for (m, n) in ((30, 50), (40, 20)):
        A = rng.standard_normal((m, n)) * (rng.random((m, n)) < 0.5)
        lp = lpgen.from_dense(A, np.zeros(n), np.zeros(m), np.zeros(m), np.zeros(n), np.ones(n))
        s = O.power_sigma_max(O.OracleLP.from_lpgen(lp))
        assert abs(s - np.linalg.norm(A, 2)) <= 1e-6 * np.linalg.norm(A, 2)


def test_power_iteration_matches_svd():
    check_power_iteration()


def check_power_rounds_by_hand():
    """The first rounds of the power iteration (reading O8) worked by hand on A = diag(3, 4):
    from v = (1, 1)/sqrt(2), w = A v = (3, 4)/sqrt(2) and lam = w^T w = 25/2; then v = A^T w /
    ||A^T w|| = (9, 16)/sqrt(337), w = (27, 64)/sqrt(337), lam = 4825/337.  With power_tol = 0
    the iteration runs exactly the given number of rounds."""
    lp = O.OracleLP(2, 2, [1.0, 1.0], [0, 1, 2], [0, 1], [3.0, 4.0], [0.0, 0.0], [1.0, 1.0],
                    [0.0, 0.0], [1.0, 1.0])
    s1 = O.power_sigma_max(lp, iters=1, tol=0.0)
    s2 = O.power_sigma_max(lp, iters=2, tol=0.0)
    assert abs(s1 - math.sqrt(25.0 / 2.0)) <= 1e-15 * s1, s1
    assert abs(s2 - math.sqrt(4825.0 / 337.0)) <= 1e-15 * s2, s2


def test_power_rounds_by_hand():
    check_power_rounds_by_hand()


def check_power_stop_rule():
    """The stopping rule |lam - lam_prev| <= tol * lam (reading O8) on A = diag(2a, a),
    a = 1000: from v = (1, 1)/sqrt(2) round k gives lam_k = a^2 (4 16^(k-1) + 1) /
    (16^(k-1) + 1) in closed form (v_k is proportional to (4^k, 1)).  The relative rule is
    blind to the scale a, so the stopping round and sigma = sqrt(lam_K) follow from exact
    fractions; a rule on the absolute change would run on far longer at this scale."""
    from fractions import Fraction as Fr

    a = 1000
    lp = O.OracleLP(2, 2, [1.0, 1.0], [0, 1, 2], [0, 1], [2.0 * a, float(a)], [0.0, 0.0],
                    [1.0, 1.0], [0.0, 0.0], [1.0, 1.0])
    lam = lambda k: Fr(a * a) * (4 * 16 ** (k - 1) + 1) / (16 ** (k - 1) + 1)
    tol, prev, k = Fr(1, 10 ** 8), Fr(0), 0
    while True:
        k += 1
        cur = lam(k)
        if abs(cur - prev) <= tol * cur:
            break
        prev = cur
    assert k == 9  # stops with a margin of about 4 on either side of the threshold
    s = O.power_sigma_max(lp)
    assert abs(s - math.sqrt(float(lam(k)))) <= 1e-14 * s, (s, math.sqrt(float(lam(k))))


def test_power_stop_rule():
    check_power_stop_rule()


def check_eta_closed_form():
    """eta = safety / sigma_max(A) (the step-size condition eta ||A||_2 < 1 of Section 2.2,
    with the documented safety factor 0.998): on A = diag(3, 4) sigma_max is 4, so
    eta = 0.998 / 4; an LP without nonzeros gets eta = 1."""
    lp = O.OracleLP(2, 2, [1.0, 1.0], [0, 1, 2], [0, 1], [3.0, 4.0], [0.0, 0.0], [1.0, 1.0],
                    [0.0, 0.0], [1.0, 1.0])
    eta = O.default_eta(lp)
    assert abs(eta - 0.998 / 4.0) <= 1e-8 * eta, eta
    empty = O.OracleLP(3, 1, [1.0, 2.0, 3.0], [0, 0], [], [], [0.0], [1.0], [0.0] * 3, [1.0] * 3)
    assert O.default_eta(empty) == 1.0


def test_eta_closed_form():
    check_eta_closed_form()


def check_default_omega():
    """omega_0 = ||c|| / ||b_fin|| (the reading of the initial primal weight): with
    c = (6, 8), ||c|| = 10, and rows '=' (b = 1, counted once), '<=' (u = 2), '>=' (l = 2),
    free, and ranged [0, 4] (two finite entries), ||b_fin||^2 = 1 + 4 + 4 + 0 + 16 = 25, so
    omega_0 = 10 / 5 = 2 exactly.  A zero cost vector or rows without finite bounds give 1."""
    lc = [1.0, -INF, 2.0, -INF, 0.0]
    uc = [1.0, 2.0, INF, INF, 4.0]
    rp = [0, 1, 2, 3, 4, 5]
    lp = O.OracleLP(2, 5, [6.0, 8.0], rp, [0, 1, 0, 1, 0], [1.0] * 5, lc, uc, [0.0, 0.0],
                    [INF, INF])
    assert O.default_omega(lp) == 2.0
    zero_c = O.OracleLP(2, 5, [0.0, 0.0], rp, [0, 1, 0, 1, 0], [1.0] * 5, lc, uc, [0.0, 0.0],
                        [INF, INF])
    assert O.default_omega(zero_c) == 1.0
    free = O.OracleLP(2, 1, [6.0, 8.0], [0, 1], [0], [1.0], [-INF], [INF], [0.0, 0.0], [1.0, 1.0])
    assert O.default_omega(free) == 1.0


def test_default_omega_hand_computed():
    check_default_omega()


def check_epoch_hand():
    """Two checks of the restarted, reflected-Halpern solve, worked by hand (Appendix B.2,
    B.3) on  min -x  s.t.  x <= 1/4,  0 <= x <= 5,  eta = 1/2, omega_0 = 1, a check after
    every iteration.

    T = 1 from (0, 0), tau = sigma = 1/2: x^ = 1/2, x_bar = 1, y^ = min(0, 0 + (1/4 - 1)/2)
    = -3/8.  P-norm of (dx, dy) = (-1/2, 3/8): 1/2 + 9/32 - 3/8 = 13/32.  First check of
    the epoch (anchor residual = r), artificial restart since k = 1 >= 0.36 T.  PID with
    d_x = 1/2, d_y = 3/8 (distances from the start): omega = d_y / d_x = 3/4.
    T = 2 from the new anchor (1/2, -3/8), tau = 2/3, sigma = 3/8: x^ = 1/2 + 5/12 = 11/12,
    x_bar = 4/3, y^ = -3/8 + (3/8)(1/4 - 4/3) = -25/32.  P-norm^2 of (-5/12, 13/32) with
    omega = 3/4: 75/288 + 169/384 - 130/384 = 139/384.  Again the epoch's first check, so
    the anchor residual is this r, and an artificial restart (k = 1 >= 0.72).  PID with the
    distances from the anchor set at T = 1: d_x = 5/12, d_y = 13/32, error log(10/13),
    integral log(4/3) + log(10/13): omega = (3/4)(13/10)(4/3)^(-0.01)."""
    lp = O.OracleLP(1, 1, [-1.0], [0, 1], [0], [1.0], [-INF], [0.25], [0.0], [5.0])
    prm = dict(eta=0.5, omega0=1.0, check_every=1)
    r1 = O.solve(lp, eps=0.0, max_iter=1, params=prm)
    assert r1.x[0] == 0.5 and r1.y[0] == -0.375
    r2 = O.solve(lp, eps=0.0, max_iter=2, params=prm)
    assert abs(r2.x[0] - 11.0 / 12.0) <= 1e-15 and abs(r2.y[0] + 25.0 / 32.0) <= 1e-15
    t0, t1 = r2.trace
    assert abs(t0["r"] - math.sqrt(13.0 / 32.0)) <= 1e-15
    assert abs(t1["r"] - math.sqrt(139.0 / 384.0)) <= 1e-14
    for t in (t0, t1):
        assert t["first"] and t["r_anchor"] == t["r"] and t["r_prev"] == t["r"]
        assert t["restart"] == 3 and t["k"] == 1
    assert t0["d_x"] == 0.5 and t0["d_y"] == 0.375
    assert abs(t1["d_x"] - 5.0 / 12.0) <= 1e-15 and abs(t1["d_y"] - 13.0 / 32.0) <= 1e-15
    assert t0["omega"] == 1.0 and abs(t1["omega"] - 0.75) <= 1e-15
    want = 0.75 * 1.3 * (4.0 / 3.0) ** -0.01
    assert abs(r2.omega - want) <= 1e-14 * want, (r2.omega, want)
    assert r2.restarts == 2


def test_epoch_bookkeeping_hand_computed():
    check_epoch_hand()


def check_epoch_trace(T=4000):
    """The restart test's inputs at every check follow their definitions (Appendix B.2,
    readings O10 and O18): an epoch's first check is the first check after a restart (or
    of the solve); its residual is the epoch's reference r(z^{n,0}) until the next restart;
    the previous-check residual is the last check's r within the epoch (the check's own r at
    the first one); the decision is the printed rule applied to those; omega changes only at
    a restart."""
    lp = lpgen.small_random_lp(4, n=300, m=150, nnz_per_col=5)
    o = O.OracleLP.from_lpgen(lp)
    res = O.solve(o, eps=0.0, max_iter=T, params=dict(check_every=16))
    tr = res.trace
    kinds = {t["restart"] for t in tr}
    assert {1, 3} <= kinds and len(tr) == T // 16, kinds  # several epochs, several kinds
    anchor = prev = None
    for i, t in enumerate(tr):
        first = i == 0 or tr[i - 1]["restart"] != 0
        assert t["first"] == first, i
        if first:
            anchor = prev = t["r"]
        assert t["r_anchor"] == anchor and t["r_prev"] == prev, i
        want = O.restart_decision(t["r"], anchor, prev, first, t["k"], t["T"], 0.2, 0.8, 0.36)
        assert t["restart"] == want, i
        prev = t["r"]
        if i and tr[i - 1]["restart"] == 0:
            assert t["omega"] == tr[i - 1]["omega"], i


def test_epoch_bookkeeping_follows_definitions():
    check_epoch_trace()


# --------------------------------------------------------------------------- restarts, PID
def check_restart_rules():
    """Appendix B.2 criteria as printed, with ties as printed (<= and >)."""
    bs, bn, ba = 0.2, 0.8, 0.36
    d = O.restart_decision
    assert d(0.2, 1.0, 0.1, False, 10, 100, bs, bn, ba) == 1  # sufficient, tie counts
    assert d(0.5, 1.0, 0.4, False, 10, 100, bs, bn, ba) == 2  # necessary: decayed, rose
    assert d(0.5, 1.0, 0.5, False, 10, 100, bs, bn, ba) == 0  # did not rise (needs >)
    assert d(0.5, 1.0, 0.4, True, 10, 100, bs, bn, ba) == 0  # not at an epoch's first check
    assert d(0.9, 1.0, 0.4, False, 10, 100, bs, bn, ba) == 0  # not decayed enough
    assert d(0.9, 1.0, 0.4, False, 36, 100, bs, bn, ba) == 3  # artificial, tie counts
    assert d(0.9, 1.0, 0.4, False, 35, 100, bs, bn, ba) == 0


def test_restart_rules():
    check_restart_rules()


def check_pid():
    """Appendix B.3: with K_P + K_I = 1 and K_D = 0 the first restart sets
    omega = d_y / d_x exactly (log omega - e = log(d_y/d_x))."""
    w, es, ep = O.pid_omega(1.0, 2.0, 1.0, 0.0, None, 0.99, 0.01, 0.0)
    assert abs(w - 0.5) <= 1e-15 and abs(es - math.log(2.0)) <= 1e-15
    w, _, _ = O.pid_omega(3.0, 1.5, 6.0, 0.0, None, 0.99, 0.01, 0.0)
    assert abs(w - 4.0) <= 4e-15
    # second restart: integral and derivative terms, evaluated by hand in logs
    e1 = math.log(2.0)
    w2, es2, e2 = O.pid_omega(0.5, 1.0, 1.0, e1, e1, 0.5, 0.25, 0.125)
    e = math.log(0.5)
    want = math.exp(math.log(0.5) - (0.5 * e + 0.25 * (e1 + e) + 0.125 * (e - e1)))
    assert abs(w2 - want) <= 1e-15 * want and abs(e2 - e) <= 1e-15
    assert O.pid_omega(2.0, 0.0, 1.0, 0.0, None, 0.99, 0.01, 0.0)[0] == 2.0  # skipped


def test_pid_primal_weight():
    check_pid()


# --------------------------------------------------------------------------- permutation
def check_permutation_invariance():
    """Permuting rows and columns changes only summation order: the oracle on a permuted
    LP, un-permuted, matches the original to 1e-12 after 100 iterations."""
    lp = lpgen.small_random_lp(2, n=300, m=150, nnz_per_col=5)
    rng = np.random.default_rng(9)
    pr, pc = rng.permutation(lp.m), rng.permutation(lp.n)
    inv_c = np.argsort(pc)
    rows = np.repeat(np.arange(lp.m), np.diff(lp.row_ptr))
    # new row i is old row pr[i]; new column j is old column pc[j]
    inv_r = np.argsort(pr)
    nr, ncl = inv_r[rows], inv_c[lp.col]
    order = np.lexsort((ncl, nr))
    rp = np.zeros(lp.m + 1, np.int64)
    np.cumsum(np.bincount(nr, minlength=lp.m), out=rp[1:])
    perm = O.OracleLP(lp.n, lp.m, lp.c[pc], rp, ncl[order], lp.val[order], lp.lc[pr], lp.uc[pr],
                      lp.lv[pc], lp.uv[pc])
    base = O.OracleLP.from_lpgen(lp)
    prm = dict(eta=0.2, check_every=32)
    a = O.solve(base, eps=0.0, max_iter=100, params=prm)
    b = O.solve(perm, eps=0.0, max_iter=100, params=prm)
    np.testing.assert_allclose(b.x[inv_c], a.x, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b.y[inv_r], a.y, rtol=1e-12, atol=1e-12)


def test_permutation_invariance():
    check_permutation_invariance()


def test_resume_from_state_is_exact():
    """Stopping at a check and resuming from the returned state reproduces the
    uninterrupted solve bit for bit."""
    lp = lpgen.small_random_lp(1, n=200, m=100, nnz_per_col=5)
    o = O.OracleLP.from_lpgen(lp)
    full = O.solve(o, eps=0.0, max_iter=256, params=dict(check_every=64))
    half = O.solve(o, eps=0.0, max_iter=128, params=dict(check_every=64))
    rest = O.solve(o, eps=0.0, max_iter=256, params=dict(check_every=64), state=half.state)
    assert np.array_equal(full.x, rest.x) and np.array_equal(full.y, rest.y)
    assert full.omega == rest.omega and full.restarts == rest.restarts


def test_diverging_step_is_reported_at_the_first_check():
    """eta far above 1 / ||A|| makes the iterates overflow; the first check must stop the
    solve with status 2 (non-finite iterate), not report convergence or run on."""
    lp = lpgen.small_random_lp(0, n=200, m=100)
    o = O.OracleLP.from_lpgen(lp)
    with np.errstate(all="ignore"):
        bad = O.solve(o, eps=1e-8, max_iter=640, params=dict(eta=1e300))
    assert bad.status == 2 and bad.iterations == 64
    ok = O.solve(o, eps=1e-4, max_iter=100_000, params=dict(eta=O.default_eta(o)))
    assert ok.status == 0


# --------------------------------------------------------------------------- check point (O11)
def check_check_point():
    """Reading O11: a check evaluates the KKT errors and the fixed-point residual at the PDHG
    output T(z) of its iteration, and a restart sets both the anchor and the iterate to T(z).
    So at a check without a restart the reported KKT values are kkt() of the returned
    (x^, y^); at a check with a restart the state continues from (x^, y^) with k = 0, and
    the next iteration is the PDHG step from (x^, y^) with the updated step sizes."""
    lp = lpgen.small_random_lp(3, n=300, m=150)
    o = O.OracleLP.from_lpgen(lp)
    prm = dict(eta=O.default_eta(o))
    kinds = [r["restart"] for r in O.solve(o, eps=0.0, max_iter=640, params=prm).trace]
    t_keep = 64 * (kinds.index(0) + 1)
    t_restart = 64 * (next(i for i, k in enumerate(kinds) if k) + 1)
    a = O.solve(o, eps=0.0, max_iter=t_keep, params=prm)
    assert a.trace[-1]["restart"] == 0
    assert a.kkt == O.kkt(o, a.x, a.y, a.eta / a.omega)
    b = O.solve(o, eps=0.0, max_iter=t_restart, params=prm)
    assert b.trace[-1]["restart"] != 0
    S = b.state
    for key in ("x", "x0"):
        assert np.array_equal(S[key], b.x), key
    for key in ("y", "y0"):
        assert np.array_equal(S[key], b.y), key
    assert S["k"] == 0
    c = O.solve(o, eps=0.0, max_iter=t_restart + 1, params=prm, state=S)
    xh, yh, _, _ = O.pdhg_step(o, b.x, b.y, b.eta / b.omega, b.eta * b.omega)
    assert np.array_equal(c.x, xh) and np.array_equal(c.y, yh)


def test_check_point_and_restart_point():
    check_check_point()
