"""Planted mistakes in the oracle must each be caught by one of its pins.

Every mutant below is a plausible slip (a dropped term, a wrong sign, a swapped bound, a
transposed operand, the garbled printed grouping of the Halpern step).  The test patches
the mutant into the oracle module on the CPU and runs the pins of
``test_oracle_pins.py``: at least one must fail.
"""
import math

import numpy as np
import pytest

from oracle import pdhg as O
import test_oracle_pins as pins

ALL_CHECKS = [
    pins.check_pdhg_hand, pins.check_dual_step_closed_forms, pins.check_halpern_fixed_point,
    pins.check_planted_optimum_is_fixed, pins.check_p_norm_dense, pins.check_kkt_hand,
    pins.check_kkt_zero_at_planted, pins.check_power_iteration, pins.check_restart_rules,
    pins.check_pid, pins.check_box_only, pins.check_knapsack,
    pins.check_eta_closed_form, pins.check_default_omega, pins.check_epoch_hand,
    lambda: pins.check_brute_force(seeds=range(2)), pins.check_epoch_trace,
    pins.check_check_point, pins.check_power_rounds_by_hand, pins.check_power_stop_rule,
]


def _orig(name):
    return getattr(O, name)


def m_primal_sign(lp, x, y, tau, sigma):
    g = lp.c + lp.ATy(y)  # wrong sign of A^T y
    xh = O.proj_X(x - tau * g, lp.lv, lp.uv)
    xbar = 2.0 * xh - x
    z = lp.Ax(xbar)
    w = y / sigma - z
    return xh, sigma * (w - O.proj_negS(w, lp.lc, lp.uc)), xbar, z


def m_no_reflection(lp, x, y, tau, sigma):
    g = lp.c - lp.ATy(y)
    xh = O.proj_X(x - tau * g, lp.lv, lp.uv)
    xbar = xh  # dropped 2 x^{k+1} - x^k
    z = lp.Ax(xbar)
    w = y / sigma - z
    return xh, sigma * (w - O.proj_negS(w, lp.lc, lp.uc)), xbar, z


def m_transposed(lp, x, y, tau, sigma):
    g = lp.c - lp.Ax(y) if lp.m == lp.n else lp.c - lp.A.T.T @ np.resize(y, lp.n)[: lp.n]
    xh = O.proj_X(x - tau * g, lp.lv, lp.uv)
    xbar = 2.0 * xh - x
    z = lp.Ax(xbar)
    w = y / sigma - z
    return xh, sigma * (w - O.proj_negS(w, lp.lc, lp.uc)), xbar, z


def m_dual_sign(lp, x, y, tau, sigma):
    g = lp.c - lp.ATy(y)
    xh = O.proj_X(x - tau * g, lp.lv, lp.uv)
    xbar = 2.0 * xh - x
    z = lp.Ax(xbar)
    w = y / sigma + z  # wrong sign of z
    return xh, sigma * (w - O.proj_negS(w, lp.lc, lp.uc)), xbar, z


def m_proj_S_not_negated(v, lc, uc):
    return np.minimum(np.maximum(v, lc), uc)


def m_halpern_printed(zh, z, z0, k, gamma):
    return (1.0 + gamma) * (k + 1.0) / (k + 2.0) * zh - gamma * z + z0 / (k + 2.0)


def m_halpern_swapped(zh, z, z0, k, gamma):
    return (1.0 / (k + 2.0)) * ((1.0 + gamma) * zh - gamma * z) + ((k + 1.0) / (k + 2.0)) * z0


def m_pnorm_sign(dx, dy, adx, omega, eta):
    return ((omega / eta) * float(np.dot(dx, dx)) + (1.0 / (eta * omega)) * float(np.dot(dy, dy))
            - 2.0 * float(np.dot(adx, dy)))


def m_pnorm_swapped(dx, dy, adx, omega, eta):
    return ((1.0 / (eta * omega)) * float(np.dot(dx, dx)) + (omega / eta) * float(np.dot(dy, dy))
            + 2.0 * float(np.dot(adx, dy)))


def _kkt_variant(rdual_tau=True, dual_obj_sign=-1.0):
    def f(lp, x, y, tau, bnorm=None, cnorm=None):
        if bnorm is None:
            bnorm = O.finite_bound_norm(lp.lc, lp.uc)
        if cnorm is None:
            cnorm = float(np.linalg.norm(lp.c))
        ax = lp.Ax(x)
        r_p = float(np.linalg.norm(ax - O.proj_S(ax, lp.lc, lp.uc))) / (1.0 + bnorm)
        g = lp.c - lp.ATy(y)
        xt = x - tau * g
        px = O.proj_X(xt, lp.lv, lp.uv)
        r_d = float(np.linalg.norm(px - x)) / (tau if rdual_tau else 1.0) / (1.0 + cnorm)
        s = (px - xt) / tau
        obj_p = float(np.dot(lp.c, x))
        obj_d = dual_obj_sign * O.p_fun(-y, lp.lc, lp.uc) + float(np.dot(s, x))
        r_g = abs(obj_p - obj_d) / (1.0 + max(abs(obj_p), abs(obj_d)))
        return dict(r_primal=r_p, r_dual=r_d, r_gap=r_g, obj_p=obj_p, obj_d=obj_d)
    return f


def m_pfun_swapped(y, l, u):
    return _orig_pfun(y, u, l)


_orig_pfun = O.p_fun


def m_pid_sign(omega, d_x, d_y, e_sum, e_prev, kp, ki, kd):
    if not (d_x > 0.0 and d_y > 0.0):
        return omega, e_sum, e_prev
    e = -math.log(math.sqrt(omega) * d_x / (d_y / math.sqrt(omega)))
    e_sum = e_sum + e
    de = 0.0 if e_prev is None else e - e_prev
    return math.exp(math.log(omega) - (kp * e + ki * e_sum + kd * de)), e_sum, e


def m_necessary_strict(r, r_anchor, r_prev, first_check, k, T, bs, bn, ba):
    if r <= bs * r_anchor:
        return 1
    if (not first_check) and r <= bn * r_anchor and r >= r_prev:
        return 2
    if k >= ba * T:
        return 3
    return 0


def m_power_no_sqrt(lp, iters=200, tol=1e-8):
    return _orig_power(lp, iters, tol) ** 2


_orig_power = O.power_sigma_max


def m_proj_X_unbounded_above(v, lv, uv):
    return np.maximum(v, lv)


def m_epoch_keeps_anchor(S):
    S["k"] = 0  # r_anchor and r_prev carried over from the epoch that ended


def m_epoch_keeps_k(S):
    S["r_anchor"] = None
    S["r_prev"] = None  # inner count k not reset


def m_distances_from_origin(xh, yh, x0, y0):
    return float(np.linalg.norm(xh)), float(np.linalg.norm(yh))


def m_omega_inverted(lp):
    cn = float(np.linalg.norm(lp.c))
    bn = O.finite_bound_norm(lp.lc, lp.uc)
    return bn / cn if (cn > 0.0 and bn > 0.0) else 1.0


def m_bound_norm_with_infinities(lc, uc):
    eq = lc == uc
    return math.sqrt(float(np.sum(np.where(eq, lc, 0.0) ** 2) + np.sum(lc[~eq] ** 2)
                           + np.sum(uc[~eq] ** 2)))


def m_eta_no_safety(lp, safety=0.998, iters=200, tol=1e-8):
    s = O.power_sigma_max(lp, iters, tol)
    return 1.0 / s if s > 0.0 else 1.0


MUTANTS = {
    "primal step sign of A^T y": ("pdhg_step", m_primal_sign),
    "dropped reflection 2x+ - x": ("pdhg_step", m_no_reflection),
    "transposed operand in primal step": ("pdhg_step", m_transposed),
    "dual step sign of z": ("pdhg_step", m_dual_sign),
    "dual projection onto S instead of -S": ("proj_negS", m_proj_S_not_negated),
    "Halpern with the printed grouping": ("halpern", m_halpern_printed),
    "Halpern weights swapped": ("halpern", m_halpern_swapped),
    "P-norm cross term sign": ("p_norm_sq", m_pnorm_sign),
    "P-norm diagonal blocks swapped": ("p_norm_sq", m_pnorm_swapped),
    "r_dual without the 1/tau": ("kkt", _kkt_variant(rdual_tau=False)),
    "dual objective sign of p(-y)": ("kkt", _kkt_variant(dual_obj_sign=1.0)),
    "p() with l and u swapped": ("p_fun", m_pfun_swapped),
    "PID error sign": ("pid_omega", m_pid_sign),
    "necessary decay with >= instead of >": ("restart_decision", m_necessary_strict),
    "power iteration returns sigma^2": ("power_sigma_max", m_power_no_sqrt),
    "box projection ignores upper bound": ("proj_X", m_proj_X_unbounded_above),
    "restart keeps the epoch's reference residual": ("new_epoch", m_epoch_keeps_anchor),
    "restart keeps the inner iteration count": ("new_epoch", m_epoch_keeps_k),
    "PID distances from the origin, not the anchor": ("anchor_distances", m_distances_from_origin),
    "omega_0 ratio inverted": ("default_omega", m_omega_inverted),
    "infinite bounds counted in ||b||": ("finite_bound_norm", m_bound_norm_with_infinities),
    "eta without the safety factor": ("default_eta", m_eta_no_safety),
}


# Slips inside the solve loop itself, planted in a copy of ``solve`` built from its source
# with one snippet replaced (the loop has no smaller function to swap).
import inspect  # noqa: E402
import textwrap  # noqa: E402

def _planted(name, old, new, module=O):
    """A copy of the oracle function ``name`` (of ``module``) built from its source with
    ``old`` replaced by ``new`` (both empty: the function itself)."""
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    assert old in src, old
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<planted {name}>", "exec"), ns)
    return ns[name]


def _solve_with(old, new):
    return _planted("solve", old, new)


SOLVE_MUTANTS = {
    "restart leaves the anchor where it was": ("            x0, y0 = xh.copy(), yh.copy()\n", ""),
    "restart continues from the Halpern iterate":
        ("            x, y = xh.copy(), yh.copy()\n            new_epoch(S)",
         "            x, y = xn, yn\n            new_epoch(S)"),
    "tau and sigma swapped": ("tau, sigma = eta / omega, eta * omega", "tau, sigma = eta * omega, eta / omega"),
    "KKT evaluated at the Halpern iterate": ("last_kkt = kkt(lp, xh, yh,", "last_kkt = kkt(lp, xn, yn,"),
    "step sizes not refreshed after the PID update":
        ("            new_epoch(S)\n            tau, sigma = eta / omega, eta * omega\n", "            new_epoch(S)\n"),
    "fixed-point residual measured from the anchor":
        ("fixed_point_residual(lp, x, y, xh, yh,", "fixed_point_residual(lp, x0, y0, xh, yh,"),
    "solution returned at the Halpern iterate": ("OracleResult(x=xh, y=yh,", "OracleResult(x=x, y=y,"),
    "artificial restart against the check count": ('S["k"], S["T"],\n', 'S["k"], S["checks"],\n'),
    "inner count not advanced": ('S["k"] = k + 1', 'S["k"] = k'),
    "check one iteration late": ('if S["T"] % K != 0 and', 'if (S["T"] - 1) % K != 0 and'),
}


def test_unplanted_solve_copy_is_the_oracle():
    """The copy built from the source, with nothing replaced, solves bit for bit as the
    oracle does, so each planted copy differs by its one snippet only."""
    import lpgen

    o = O.OracleLP.from_lpgen(lpgen.small_random_lp(3, n=300, m=150))
    a = _solve_with("", "")(o, eps=0.0, max_iter=300)
    b = O.solve(o, eps=0.0, max_iter=300)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y) and a.trace == b.trace


@pytest.mark.parametrize("name", sorted(SOLVE_MUTANTS))
def test_solve_mutant_is_caught(name, monkeypatch):
    monkeypatch.setattr(O, "solve", _solve_with(*SOLVE_MUTANTS[name]))
    caught = None
    with np.errstate(all="ignore"):
        for check in ALL_CHECKS:
            try:
                check()
            except Exception as e:
                caught = (getattr(check, "__name__", "check"), type(e).__name__)
                break
    assert caught, f"no pin caught the planted mistake: {name}"


# Slips inside the KKT formulas (Appendix B.4), planted the same way in copies of ``kkt``.
def _kkt_with(old, new):
    return _planted("kkt", old, new)


KKT_MUTANTS = {
    "r_primal without the 1 + in its denominator":
        ("r_p = float(np.linalg.norm(rp_vec)) / (1.0 + bnorm)",
         "r_p = float(np.linalg.norm(rp_vec)) / max(bnorm, 1e-300)"),
    "r_primal normalised by ||c||":
        ("r_p = float(np.linalg.norm(rp_vec)) / (1.0 + bnorm)",
         "r_p = float(np.linalg.norm(rp_vec)) / (1.0 + cnorm)"),
    "r_dual without the 1 + in its denominator": ("/ tau / (1.0 + cnorm)", "/ tau / max(cnorm, 1e-300)"),
    "gap denominator with min": ("(1.0 + max(abs(obj_p), abs(obj_d)))", "(1.0 + min(abs(obj_p), abs(obj_d)))"),
    "reduced cost s with its sign flipped": ("s = (px - xt) / tau", "s = (xt - px) / tau"),
    "dual objective without s^T x": ("+ float(np.dot(s, x)) - 0.5 * quad", "- 0.5 * quad"),
    "primal residual against -S": ("rp_vec = ax - proj_S(ax, lp.lc, lp.uc)",
                                   "rp_vec = ax + proj_negS(ax, lp.lc, lp.uc)"),
}


def test_unplanted_kkt_copy_is_the_oracle():
    import lpgen

    lp = lpgen.small_random_lp(3, n=300, m=150)
    o = O.OracleLP.from_lpgen(lp)
    x, y = lp.x_star + 0.1, lp.y_star - 0.2
    assert _kkt_with("", "")(o, x, y, 0.3) == O.kkt(o, x, y, 0.3)


@pytest.mark.parametrize("name", sorted(KKT_MUTANTS))
def test_kkt_mutant_is_caught(name, monkeypatch):
    monkeypatch.setattr(O, "kkt", _kkt_with(*KKT_MUTANTS[name]))
    caught = None
    with np.errstate(all="ignore"):
        for check in ALL_CHECKS:
            try:
                check()
            except Exception as e:
                caught = (getattr(check, "__name__", "check"), type(e).__name__)
                break
    assert caught, f"no pin caught the planted mistake: {name}"


# Slips inside the PDHG step (Section 2.2), the Halpern step (Appendix B.1), the restart
# rules (Appendix B.2) and the PID update (Appendix B.3).
RULE_MUTANTS = {
    "extrapolation 2 x^ + x": ("pdhg_step", "xbar = 2.0 * xh - x", "xbar = 2.0 * xh + x"),
    "dual argument y * sigma": ("pdhg_step", "w = y / sigma - z", "w = y * sigma - z"),
    "dual step without the sigma factor": ("pdhg_step", "yh = sigma * (w - proj_negS(w, lp.lc, lp.uc))",
                                           "yh = (w - proj_negS(w, lp.lc, lp.uc))"),
    "dual box with its bounds swapped": ("pdhg_step", "proj_negS(w, lp.lc, lp.uc)", "proj_negS(w, lp.uc, lp.lc)"),
    "primal step with sigma": ("pdhg_step", "xh = proj_X(x - tau * g, lp.lv, lp.uv)",
                               "xh = proj_X(x - sigma * g, lp.lv, lp.uv)"),
    "reflection with 1 - gamma": ("halpern", "((1.0 + gamma) * zh - gamma * z)", "((1.0 - gamma) * zh + gamma * z)"),
    "Halpern weight k / (k + 1)": ("halpern", "w1 = (k + 1.0) / (k + 2.0)", "w1 = k / (k + 1.0)"),
    "anchor weight 1 / (k + 1)": ("halpern", "w0 = 1.0 / (k + 2.0)", "w0 = 1.0 / (k + 1.0)"),
    "power iteration from an unnormalised start":
        ("power_sigma_max", "v = np.full(n, 1.0 / math.sqrt(n))", "v = np.full(n, 1.0)"),
    "power iteration from 1/n": ("power_sigma_max", "v = np.full(n, 1.0 / math.sqrt(n))", "v = np.full(n, 1.0 / n)"),
    "Rayleigh quotient as ||A v||": ("power_sigma_max", "lam = float(np.dot(w, w))", "lam = float(np.linalg.norm(w))"),
    "power iteration stops on the absolute change":
        ("power_sigma_max", "if abs(lam - lam_prev) <= tol * lam:", "if abs(lam - lam_prev) <= tol:"),
    "equality rows counted twice in ||b||":
        ("finite_bound_norm", "eq = np.isfinite(lc) & np.isfinite(uc) & (lc == uc)",
         "eq = np.zeros_like(lc, dtype=bool)"),
    "p() without its lower-bound term": ("p_fun", "return float(np.sum(tu) - np.sum(tl))", "return float(np.sum(tu))"),
    "p() with its lower-bound term added": ("p_fun", "return float(np.sum(tu) - np.sum(tl))",
                                            "return float(np.sum(tu) + np.sum(tl))"),
    "p() forming 0 * inf": ("p_fun", "    nz = yp > 0\n    tu[nz] = u[nz] * yp[nz]\n    nz = ym > 0\n"
                                     "    tl[nz] = l[nz] * ym[nz]", "    tu = u * yp\n    tl = l * ym"),
    "projection onto -S with its bounds swapped":
        ("proj_negS", "return np.minimum(np.maximum(v, -uc), -lc)", "return np.minimum(np.maximum(v, -lc), -uc)"),
    "necessary decay allowed at the epoch's first check":
        ("restart_decision", "if (not first_check) and r <=", "if r <="),
    "sufficient decay with <": ("restart_decision", "if r <= beta_s * r_anchor:", "if r < beta_s * r_anchor:"),
    "artificial restart with >": ("restart_decision", "if k >= beta_a * T:", "if k > beta_a * T:"),
    "artificial restart against a fixed length": ("restart_decision", "if k >= beta_a * T:", "if k >= beta_a * 64:"),
    "necessary decay against beta_sufficient":
        ("restart_decision", "r <= beta_n * r_anchor and", "r <= beta_s * r_anchor and"),
    "PID integral without the current error": ("pid_omega", "e_sum = e_sum + e", "e_sum = e_sum"),
    "PID derivative sign": ("pid_omega", "de = 0.0 if e_prev is None else (e - e_prev)",
                            "de = 0.0 if e_prev is None else (e_prev - e)"),
    "PID error without the sqrt(omega) weights":
        ("pid_omega", "e = math.log((so * d_x) / (d_y / so))", "e = math.log(d_x / d_y)"),
}


@pytest.mark.parametrize("name", sorted(RULE_MUTANTS))
def test_rule_mutant_is_caught(name, monkeypatch):
    fn, old, new = RULE_MUTANTS[name]
    monkeypatch.setattr(O, fn, _planted(fn, old, new))
    caught = None
    with np.errstate(all="ignore"):
        for check in ALL_CHECKS:
            try:
                check()
            except Exception as e:
                caught = (getattr(check, "__name__", "check"), type(e).__name__)
                break
    assert caught, f"no pin caught the planted mistake: {name}"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(O, attr, fn)
    caught = None
    for check in ALL_CHECKS:  # cheapest first; one failing pin is enough
        try:
            check()
        except Exception as e:  # AssertionError, or a shape error from a wrong operand
            caught = (getattr(check, "__name__", "check"), type(e).__name__)
            break
    assert caught, f"no pin caught the planted mistake: {name}"


# ----------------------------------------------------------------------------- diagonal QP
# Plausible slips in the QP variant (Section "Extensions to Diagonal QPs"), each caught by
# one of the QP pins of ``test_qp_oracle.py`` (the prox step by hand, the separable box QP's
# closed form, the KKT values at an equality QP's optimum, ...).
import test_qp_oracle as qpins  # noqa: E402

QP_CHECKS = [qpins.test_prox_step_by_hand, qpins.test_separable_box_qp_closed_form,
             qpins.test_equality_qp_matches_kkt_system, qpins.test_bounded_qp_matches_slsqp]


def _qp_step_variant(tau_in_prox=True, clamp_first=False):
    def f(lp, x, y, tau, sigma):
        g = lp.c - lp.ATy(y)
        if lp.q is None:
            xh = O.proj_X(x - tau * g, lp.lv, lp.uv)
        else:
            den = 1.0 + (tau if tau_in_prox else 1.0) * lp.q
            xh = (O.proj_X(x - tau * g, lp.lv, lp.uv) / den if clamp_first
                  else O.proj_X((x - tau * g) / den, lp.lv, lp.uv))
        xbar = 2.0 * xh - x
        z = lp.Ax(xbar)
        w = y / sigma - z
        return xh, sigma * (w - O.proj_negS(w, lp.lc, lp.uc)), xbar, z
    return f


def _qp_kkt_variant(grad_has_qx=True, dual_quad=-0.5, primal_quad=0.5):
    def f(lp, x, y, tau, bnorm=None, cnorm=None, row_w=None, col_w=None):
        if bnorm is None:
            bnorm = O.finite_bound_norm(lp.lc, lp.uc)
        if cnorm is None:
            cnorm = float(np.linalg.norm(lp.c))
        ax = lp.Ax(x)
        quad = 0.0 if lp.q is None else float(np.dot(lp.q * x, x))
        rp = ax - O.proj_S(ax, lp.lc, lp.uc)
        if row_w is not None:
            rp = rp * row_w
        r_p = float(np.linalg.norm(rp)) / (1.0 + bnorm)
        g = lp.c + lp.q * x - lp.ATy(y) if (lp.q is not None and grad_has_qx) else lp.c - lp.ATy(y)
        xt = x - tau * g
        px = O.proj_X(xt, lp.lv, lp.uv)
        rd = px - x
        if col_w is not None:
            rd = rd * col_w
        r_d = float(np.linalg.norm(rd)) / tau / (1.0 + cnorm)
        s = (px - xt) / tau
        obj_p = float(np.dot(lp.c, x)) + primal_quad * quad
        obj_d = -O.p_fun(-y, lp.lc, lp.uc) + float(np.dot(s, x)) + dual_quad * quad
        r_g = abs(obj_p - obj_d) / (1.0 + max(abs(obj_p), abs(obj_d)))
        return dict(r_primal=r_p, r_dual=r_d, r_gap=r_g, obj_p=obj_p, obj_d=obj_d)
    return f


QP_MUTANTS = {
    "QP prox step without tau": ("pdhg_step", _qp_step_variant(tau_in_prox=False)),
    "QP prox step clamped before the division": ("pdhg_step", _qp_step_variant(clamp_first=True)),
    "QP dual residual without Q x in the gradient": ("kkt", _qp_kkt_variant(grad_has_qx=False)),
    "QP dual objective adds 1/2 x^T Q x": ("kkt", _qp_kkt_variant(dual_quad=0.5)),
    "QP primal objective without the 1/2": ("kkt", _qp_kkt_variant(primal_quad=1.0)),
}


def test_qp_kkt_and_step_variants_match_the_oracle():
    """The unmutated variants reproduce the oracle's QP step and KKT exactly, so each mutant
    above differs from the oracle by its one planted change only."""
    o = qpins.qp(np.array([[1.0, 2.0], [0.0, 1.0]]), [1.0, -1.0], [0.0, -np.inf], [1.0, 2.0],
                 [0.0, -1.0], [3.0, np.inf], [0.5, 2.0])
    x, y = np.array([0.3, -0.2]), np.array([0.1, -0.4])
    assert all(np.array_equal(a, b) for a, b in
               zip(_qp_step_variant()(o, x, y, 0.3, 0.7), O.pdhg_step(o, x, y, 0.3, 0.7)))
    assert _qp_kkt_variant()(o, x, y, 0.3) == O.kkt(o, x, y, 0.3)


@pytest.mark.parametrize("name", sorted(QP_MUTANTS))
def test_qp_mutant_is_caught(name, monkeypatch):
    attr, fn = QP_MUTANTS[name]
    monkeypatch.setattr(O, attr, fn)
    caught = None
    for check in QP_CHECKS:
        try:
            check()
        except Exception as e:
            caught = (check.__name__, type(e).__name__)
            break
    assert caught, f"no pin caught the planted mistake: {name}"


# ----------------------------------------------------------------------------- preconditioning
# Plausible slips in the optional preconditioning (reading O15), each caught by one of the
# pins of ``test_precond_oracle.py``.
import scipy.sparse as sp  # noqa: E402

from oracle import precond as P  # noqa: E402
import test_precond_oracle as ppins  # noqa: E402

PRECOND_CHECKS = [ppins.test_pow2_nearest, ppins.test_factors_are_powers_of_two_and_scaling_is_exact,
                  ppins.test_ruiz_equilibrates, ppins.test_kkt_is_reported_for_the_original_lp,
                  ppins.test_identity_scaling_is_the_plain_solve,
                  ppins.test_preconditioned_solve_reaches_planted_optimum,
                  ppins.test_preconditioned_answer_satisfies_the_original_kkt]

_orig_scaled_lp = P.scaled_lp
_orig_precond_solve = P.solve
_orig_pow2 = P.pow2_nearest


def _scaled_variant(bounds="div", rows="mul", cost="mul"):
    def f(lp, dr, dc):
        A = (sp.diags(dr) @ lp.A @ sp.diags(dc)).tocsr()
        A.sort_indices()
        rw = dr if rows == "mul" else 1.0 / dr
        cc = dc * lp.c if cost == "mul" else lp.c / dc
        lv, uv = (lp.lv / dc, lp.uv / dc) if bounds == "div" else (lp.lv * dc, lp.uv * dc)
        return O.OracleLP(lp.n, lp.m, cc, A.indptr, A.indices, A.data, rw * lp.lc, rw * lp.uc,
                          lv, uv, None if lp.q is None else dc * dc * lp.q)
    return f


def _precond_solve_variant(y_back="mul", weights="inv"):
    def f(lp, eps=1e-8, max_iter=100_000, params=None, x_start=None, y_start=None,
          ruiz_passes=10, pock_chambolle=True):
        dr, dc = P.scale_factors(lp, ruiz_passes, pock_chambolle)
        S = P.scaled_lp(lp, dr, dc)
        wr, wc = (1.0 / dr, 1.0 / dc) if weights == "inv" else (dr, dc)
        w = (wr, wc, O.finite_bound_norm(lp.lc, lp.uc), float(np.linalg.norm(lp.c)))
        res = O.solve(S, eps, max_iter, params,
                      None if x_start is None else np.asarray(x_start) / dc,
                      None if y_start is None else np.asarray(y_start) / dr, kkt_weights=w)
        res.x = dc * res.x
        res.y = dr * res.y if y_back == "mul" else res.y / dr
        return res
    return f


def m_ruiz_without_sqrt(norms):
    norms = np.asarray(norms, np.float64).ravel()
    out = np.ones_like(norms)
    pos = norms > 0
    out[pos] = _orig_pow2(1.0 / norms[pos])
    return out


def m_pow2_arithmetic_midpoint(v):
    m, e = np.frexp(np.asarray(v, np.float64))
    return np.ldexp(1.0, np.where(m >= 0.75, e, e - 1))


PRECOND_MUTANTS = {
    "scaled variable bounds multiplied by D_c": ("scaled_lp", _scaled_variant(bounds="mul")),
    "scaled row bounds divided by D_r": ("scaled_lp", _scaled_variant(rows="div")),
    "scaled cost divided by D_c": ("scaled_lp", _scaled_variant(cost="div")),
    "dual answer divided by D_r on the way back": ("solve", _precond_solve_variant(y_back="div")),
    "KKT weights D_r, D_c instead of their inverses": ("solve", _precond_solve_variant(weights="dir")),
    "Ruiz factor without the square root": ("_factors", m_ruiz_without_sqrt),
    "power-of-two rounding at the arithmetic midpoint": ("pow2_nearest", m_pow2_arithmetic_midpoint),
}


def test_precond_variants_match_the_oracle():
    """The unmutated variants reproduce the oracle's scaled LP and preconditioned solve
    exactly, so each mutant differs from the oracle by its one planted change only."""
    import lpgen

    o = O.OracleLP.from_lpgen(lpgen.small_random_lp(2, n=120, m=60))
    dr, dc = P.scale_factors(o)
    a, b = _scaled_variant()(o, dr, dc), _orig_scaled_lp(o, dr, dc)
    for k in ("c", "lc", "uc", "lv", "uv"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    ra, rb = _precond_solve_variant()(o, 0.0, 100), _orig_precond_solve(o, 0.0, 100)
    assert np.array_equal(ra.x, rb.x) and np.array_equal(ra.y, rb.y) and ra.kkt == rb.kkt


@pytest.mark.parametrize("name", sorted(PRECOND_MUTANTS))
def test_precond_mutant_is_caught(name, monkeypatch):
    attr, fn = PRECOND_MUTANTS[name]
    monkeypatch.setattr(P, attr, fn)
    caught = None
    with np.errstate(all="ignore"):  # a planted slip may make the solve overflow
        for check in PRECOND_CHECKS:
            try:
                check()
            except Exception as e:
                caught = (check.__name__, type(e).__name__)
                break
    assert caught, f"no pin caught the planted mistake: {name}"


# ----------------------------------------------------------------------------- warm-start network
# Slips in the network's forward pass, each caught by a forward pin of ``test_gnn_oracle.py``
# (closed forms and invariants).  The finite-difference pins are left out here: a slip made
# the same way in the forward and the backward pass would pass them.
from oracle import gnn as G  # noqa: E402
import test_gnn_oracle as gpins  # noqa: E402

GNN_FORWARD_CHECKS = [gpins.test_aggregation_by_hand, gpins.test_zero_weights_closed_form,
                      gpins.test_routed_channel_closed_form, gpins.test_no_messages_is_node_local,
                      gpins.test_components_are_independent, gpins.test_permutation_equivariance]

_orig_gnn_forward = G.forward
_orig_aggregation = G.aggregation


def _forward_variant(stale_constraints=False, relu_constraints=True, head_first=False, rounds=None):
    def f(theta, R, C, Fv, Fc):
        P = G.unpack(np.asarray(theta, np.float64))
        hv = G.relu(Fv @ P["Ev"].T + P["ev"])
        hc = G.relu(Fc @ P["Ec"].T + P["ec"])
        hv0, hc0 = hv, hc
        cache = {"hv": [hv], "hc": [hc], "gv": [], "gc": []}
        for l in range(G.L if rounds is None else rounds):
            gc = R @ hv
            zc = hc @ P[f"Uc{l}"].T + gc @ P[f"Vc{l}"].T + P[f"bc{l}"]
            hc_new = G.relu(zc) if relu_constraints else zc
            gv = C @ (hc if stale_constraints else hc_new)
            hc = hc_new
            hv = G.relu(hv @ P[f"Uv{l}"].T + gv @ P[f"Vv{l}"].T + P[f"bv{l}"])
            cache["gc"].append(gc)
            cache["hc"].append(hc)
            cache["gv"].append(gv)
            cache["hv"].append(hv)
        hx, hy = (hv0, hc0) if head_first else (hv, hc)
        return hx @ P["wx"] + P["bx"], hy @ P["wy"] + P["by"], cache
    return f


def _aggregation_variant(by_count=False, swapped=False):
    def f(n, m, row_ptr, col, val):
        A = sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(row_ptr)),
                          shape=(m, n))
        W = (A != 0).astype(np.float64) if by_count else abs(A)
        rs = np.maximum(1.0, np.asarray(W.sum(axis=1)).ravel())
        cs = np.maximum(1.0, np.asarray(W.sum(axis=0)).ravel())
        if swapped:  # each side normalised by the other side's sums
            return (A @ sp.diags(1.0 / cs)).tocsr(), (A.T @ sp.diags(1.0 / rs)).tocsr()
        return (sp.diags(1.0 / rs) @ A).tocsr(), (sp.diags(1.0 / cs) @ A.T).tocsr()
    return f


GNN_MUTANTS = {
    "variable update reads the constraint state from before the round":
        ("forward", _forward_variant(stale_constraints=True)),
    "no ReLU in the constraint update": ("forward", _forward_variant(relu_constraints=False)),
    "heads read the encoder output, not the last round": ("forward", _forward_variant(head_first=True)),
    "one message-passing round too few": ("forward", _forward_variant(rounds=G.L - 1)),
    "aggregation normalised by neighbour counts": ("aggregation", _aggregation_variant(by_count=True)),
    "aggregation normalised by the other side's sums": ("aggregation", _aggregation_variant(swapped=True)),
}


def test_gnn_variants_match_the_oracle():
    """The unmutated variants reproduce the oracle's forward pass and aggregation exactly."""
    rng, A, R, C, Fv, Fc, _, _ = gpins.setup(3)
    th = gpins.random_theta(rng)
    a, b = _forward_variant()(th, R, C, Fv, Fc), _orig_gnn_forward(th, R, C, Fv, Fc)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for p, q in zip(_aggregation_variant()(A.shape[1], A.shape[0], A.indptr, A.indices, A.data),
                    _orig_aggregation(A.shape[1], A.shape[0], A.indptr, A.indices, A.data)):
        assert (p != q).nnz == 0


@pytest.mark.parametrize("name", sorted(GNN_MUTANTS))
def test_gnn_mutant_is_caught(name, monkeypatch):
    attr, fn = GNN_MUTANTS[name]
    monkeypatch.setattr(G, attr, fn)
    caught = None
    for check in GNN_FORWARD_CHECKS:
        try:
            check()
        except Exception as e:
            caught = (check.__name__, type(e).__name__)
            break
    assert caught, f"no forward pin caught the planted mistake: {name}"


# Slips in the network's backward pass, each caught by the finite-difference pins (every bias
# and head entry, and entries of every weight block).
GNN_FD_CHECKS = [lambda: gpins.test_gradient_matches_finite_differences(0),
                 lambda: gpins.test_gradient_matches_finite_differences(1)]

GNN_BACKWARD_MUTANTS = {
    "a weight gradient transposed": ('G[f"Uv{l}"] = dz.T @ K["hv"][l]', 'G[f"Uv{l}"] = (dz.T @ K["hv"][l]).T'),
    "ReLU mask of the round's input": ('dz = dhv * (K["hv"][l + 1] > 0)', 'dz = dhv * (K["hv"][l] > 0)'),
    "message gradient through C^T dropped": ("dhc = dhc + C.T @ dgv", "dhc = dhc"),
    "message gradient through R^T dropped": ("dhv = dhv + R.T @ dgc", "dhv = dhv"),
    "Vc gradient from the next round's messages":
        ('G[f"Vc{l}"] = dz.T @ K["gc"][l]', 'G[f"Vc{l}"] = dz.T @ K["gc"][min(l + 1, L - 1)]'),
    "encoder gradient without its ReLU mask": ('dz = dhv * (K["hv"][0] > 0)\n    G["Ev"]', 'dz = dhv\n    G["Ev"]'),
    "loss gradient without the 1/n": ("dx = 2.0 * (x_hat - tx) / n", "dx = 2.0 * (x_hat - tx)"),
    "encoder gradient against permuted features": ('G["Ec"] = dz.T @ Fc', 'G["Ec"] = dz.T @ Fc[::-1]'),
}


def test_unplanted_backward_copy_is_the_oracle():
    rng, A, R, C, Fv, Fc, tx, ty = gpins.setup(4)
    th = gpins.random_theta(rng)
    a = _planted("backward", "", "", module=G)(th, R, C, Fv, Fc, tx, ty)
    b = G.backward(th, R, C, Fv, Fc, tx, ty)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("name", sorted(GNN_BACKWARD_MUTANTS))
def test_gnn_backward_mutant_is_caught(name, monkeypatch):
    monkeypatch.setattr(G, "backward", _planted("backward", *GNN_BACKWARD_MUTANTS[name], module=G))
    caught = None
    for check in GNN_FD_CHECKS:
        try:
            check()
        except Exception as e:
            caught = type(e).__name__
            break
    assert caught, f"no pin caught the planted mistake: {name}"
