"""FP64 CPU oracle for restarted, reflected-Halpern PDHG on a sparse LP.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
and reference legs of ``bench.py`` may import this module.  The product path (the CUDA
library and its Python binding) never calls it, and this module shares no code with it.

It restates, step by step and in the paper's order and notation, the method of
"D-PDLP: Scaling PDLP to Distributed Multi-GPU Systems" (arXiv 2601.07628) on one device:

* the LP and its saddle point, Section 2.1 (Eq. prob:primal, Eq. prob:saddle), with the
  dual set Y of the same section;
* the PDHG step, Section 2.2 (the update rules for x^{k+1} and y^{k+1}), with the step
  sizes tau = eta / omega and sigma = eta * omega;
* the reflected Halpern step, Appendix B.1 (also step 3 of Algorithm 1);
* the fixed-point residual in the P-norm, Appendix B (the metric P) and Appendix D.2.1;
* adaptive restarts, Appendix B.2; the PID primal weight, Appendix B.3 and D.2.2;
* the relative KKT error and the dual problem, Appendix B.4 and D.1.

Arithmetic is IEEE binary64 throughout.  Sparse products use scipy's CSR kernels, which
sum each row left to right in stored order; norms and dots use numpy.

Readings of passages the paper leaves open (the same readings the CUDA path takes):

* Lagrangian sign: L = c^T x - y^T A x - p(-y; lc, uc), the only sign consistent with the
  PDHG step (c - A^T y) and the dual constraint c - A^T y = r.
* Dual step: z^{k+1} is A(2 x^{k+1} - x^k) (Algorithm 1, step 2).  The step is evaluated
  as sigma * (w - proj_{-S}(w)) with w = y^k / sigma - z, which is the printed expression
  with y^k - sigma z written as sigma * w; in this form the result lies in Y exactly.
* Halpern weights: z^{k+1} = ((k+1)/(k+2)) ((1+gamma) PDHG(z^k) - gamma z^k) + z^0/(k+2),
  whose weights sum to one (the printed grouping does not, and would not keep a fixed
  point fixed); k counts iterations since the last restart.
* Start point x = proj_X(0), y = 0; eta = 0.998 / sigma_max(A) from power iteration on
  A^T A (eta = 1 when A has no nonzeros); omega_0 = ||c|| / ||b_fin|| (1 if either is 0).
* KKT at the PDHG output (x^, y^) of each check iteration, every ``check_every`` = 64
  iterations; ||[lc, uc]|| taken over the finite entries, an equality row counted once;
  the dual objective is -p(-y) + s^T x exactly as printed; terms 0 * inf of p() vanish.
* Restart reference r(z^{n,0}) is the residual at the first check of the epoch; the
  necessary-decay test compares with the previous check of the same epoch and is not
  applied at an epoch's first check; a restart sets anchor and iterate to (x^, y^).
* PID: the derivative term is zero at the first restart; the update is skipped when
  d_x or d_y is zero or not finite.

Parity unpinned: the numeric values of the restart thresholds (beta_sufficient = 0.2,
beta_necessary = 0.8, beta_artificial = 0.36), of the PID gains (K_P = 0.99, K_I = 0.01,
K_D = 0) and of the step-size safety factor (0.998) are not given by the paper; nothing but
agreement with the CUDA path pins them.  The decision rules, the epoch bookkeeping, the PID
formula and distances, omega_0 and eta = safety / sigma_max are pinned by tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

DEFAULTS = dict(
    eta=None,  # None: 0.998 / sigma_max(A) by power iteration
    eta_safety=0.998,
    power_iters=200,
    power_tol=1e-8,
    omega0=None,  # None: ||c|| / ||b_fin||
    gamma=1.0,  # reflection coefficient of the Halpern step
    halpern=1,  # 0: plain PDHG, z^{k+1} = PDHG(z^k)
    check_every=64,
    restart=1,
    beta_sufficient=0.2,
    beta_necessary=0.8,
    beta_artificial=0.36,
    pid=1,
    pid_kp=0.99,
    pid_ki=0.01,
    pid_kd=0.0,
)


# ----------------------------------------------------------------------------- problem data
class OracleLP:
    """LP of Eq. prob:primal: min c^T x, lc <= A x <= uc, lv <= x <= uv (CSR input).

    With ``q`` (the diagonal of a positive semidefinite Q, Section "Extensions to Diagonal
    QPs") the objective is 1/2 x^T Q x + c^T x: the diagonal QP the same iteration solves."""

    def __init__(self, n, m, c, row_ptr, col, val, lc, uc, lv, uv, q=None):
        self.n, self.m = int(n), int(m)
        self.q = None if q is None else np.asarray(q, dtype=np.float64).copy()
        self.c = np.asarray(c, dtype=np.float64).copy()
        self.lc = np.asarray(lc, dtype=np.float64).copy()
        self.uc = np.asarray(uc, dtype=np.float64).copy()
        self.lv = np.asarray(lv, dtype=np.float64).copy()
        self.uv = np.asarray(uv, dtype=np.float64).copy()
        self.A = sp.csr_matrix(
            (np.asarray(val, dtype=np.float64), np.asarray(col, dtype=np.int64),
             np.asarray(row_ptr, dtype=np.int64)), shape=(self.m, self.n))
        # A^T stored row-wise: each column of A summed in stored (row) order.
        self.AT = self.A.T.tocsr()
        self.AT.sort_indices()

    @classmethod
    def from_lpgen(cls, lp):
        return cls(lp.n, lp.m, lp.c, lp.row_ptr, lp.col, lp.val, lp.lc, lp.uc, lp.lv, lp.uv)

    def Ax(self, x):
        return self.A @ x

    def ATy(self, y):
        return self.AT @ y


# ----------------------------------------------------------------------------- projections
def proj_X(v, lv, uv):
    """Projection onto X = {lv <= x <= uv} (Section 2.1): a per-element clamp."""
    return np.minimum(np.maximum(v, lv), uv)


def proj_S(v, lc, uc):
    """Projection onto S = {lc <= s <= uc} (Section 2.1)."""
    return np.minimum(np.maximum(v, lc), uc)


def proj_negS(v, lc, uc):
    """Projection onto -S = {-uc <= s <= -lc} (Section 2.2, dual update)."""
    return np.minimum(np.maximum(v, -uc), -lc)


def p_fun(y, l, u):
    """p(y; l, u) = u^T y^+ - l^T y^- (Section 2.1), a term being 0 when its multiplier
    y^+ or y^- is 0 (so 0 * inf contributes nothing)."""
    yp = np.maximum(y, 0.0)
    ym = np.maximum(-y, 0.0)
    tu = np.zeros_like(y)
    tl = np.zeros_like(y)
    nz = yp > 0
    tu[nz] = u[nz] * yp[nz]
    nz = ym > 0
    tl[nz] = l[nz] * ym[nz]
    return float(np.sum(tu) - np.sum(tl))


def finite_bound_norm(lc, uc):
    """||[lc, uc]||_2 over the finite entries, an equality row (lc == uc) counted once."""
    eq = np.isfinite(lc) & np.isfinite(uc) & (lc == uc)
    tot = np.sum(np.where(eq, lc, 0.0) ** 2)
    lfin = np.isfinite(lc) & ~eq
    ufin = np.isfinite(uc) & ~eq
    tot += np.sum(lc[lfin] ** 2) + np.sum(uc[ufin] ** 2)
    return math.sqrt(tot)


# ----------------------------------------------------------------------------- step size
def power_sigma_max(lp: OracleLP, iters=200, tol=1e-8):
    """Largest singular value of A by power iteration on A^T A.

    Start v = 1/sqrt(n) in every entry; each round computes w = A v, the Rayleigh quotient
    lam = w^T w (v has unit norm), then v <- A^T w / ||A^T w||; stop after ``iters`` rounds
    or when |lam - lam_prev| <= tol * lam.  Returns sqrt(lam) (0 when A v vanishes)."""
    n = lp.n
    if n == 0 or lp.A.nnz == 0:
        return 0.0
    v = np.full(n, 1.0 / math.sqrt(n))
    lam_prev = 0.0
    lam = 0.0
    for _ in range(iters):
        w = lp.Ax(v)
        lam = float(np.dot(w, w))
        u = lp.ATy(w)
        un = float(np.linalg.norm(u))
        if un == 0.0 or lam == 0.0:
            return math.sqrt(lam)
        v = u / un
        if abs(lam - lam_prev) <= tol * lam:
            break
        lam_prev = lam
    return math.sqrt(lam)


def default_eta(lp: OracleLP, safety=0.998, iters=200, tol=1e-8):
    s = power_sigma_max(lp, iters, tol)
    return safety / s if s > 0.0 else 1.0


def default_omega(lp: OracleLP):
    cn = float(np.linalg.norm(lp.c))
    bn = finite_bound_norm(lp.lc, lp.uc)
    return cn / bn if (cn > 0.0 and bn > 0.0) else 1.0


# ----------------------------------------------------------------------------- PDHG step
def pdhg_step(lp: OracleLP, x, y, tau, sigma):
    """One PDHG step (Section 2.2; Algorithm 1, steps 1-2).

    x^{k+1} = proj_X(x^k - tau (c - A^T y^k))
    y^{k+1} = y^k - sigma z - sigma proj_{-S}(y^k / sigma - z),   z = A (2 x^{k+1} - x^k)

    Returns (x^, y^, x_bar, z)."""
    g = lp.c - lp.ATy(y)
    if lp.q is None:
        xh = proj_X(x - tau * g, lp.lv, lp.uv)
    else:  # diagonal QP (Eq. primal_update): per coordinate a clamped 1-D quadratic minimum
        xh = proj_X((x - tau * g) / (1.0 + tau * lp.q), lp.lv, lp.uv)
    xbar = 2.0 * xh - x
    z = lp.Ax(xbar)
    w = y / sigma - z
    yh = sigma * (w - proj_negS(w, lp.lc, lp.uc))
    return xh, yh, xbar, z


def halpern(zh, z, z0, k, gamma):
    """Reflected Halpern step (Appendix B.1; Algorithm 1, step 3):
    z^{k+1} = ((k+1)/(k+2)) ((1+gamma) PDHG(z^k) - gamma z^k) + z^0 / (k+2)."""
    w1 = (k + 1.0) / (k + 2.0)
    w0 = 1.0 / (k + 2.0)
    return w1 * ((1.0 + gamma) * zh - gamma * z) + w0 * z0


# ----------------------------------------------------------------------------- residuals
def kkt(lp: OracleLP, x, y, tau, bnorm=None, cnorm=None, row_w=None, col_w=None):
    """Relative KKT errors of Appendix B.4 at (x, y), with the current primal step tau.

    r_primal = ||Ax - proj_S(Ax)|| / (1 + ||[lc, uc]||)
    r_dual   = ||proj_X(x - tau (c - A^T y)) - x|| / tau / (1 + ||c||)
    r_gap    = |c^T x + p(-y) - s^T x| / (1 + max(|c^T x|, |-p(-y) + s^T x|))
    s        = (proj_X(x - tau (c - A^T y)) - (x - tau (c - A^T y))) / tau

    ``row_w`` and ``col_w`` (optional) weight the entries of the primal and dual residual
    vectors: for an LP scaled as D_r A D_c they are 1 / D_r and 1 / D_c, which turns the
    residuals of the scaled LP into those of the original one (the objectives are the same
    in both); ``bnorm`` and ``cnorm`` are then the original LP's.
    """
    if bnorm is None:
        bnorm = finite_bound_norm(lp.lc, lp.uc)
    if cnorm is None:
        cnorm = float(np.linalg.norm(lp.c))
    ax = lp.Ax(x)
    quad = 0.0 if lp.q is None else float(np.dot(lp.q * x, x))  # x^T Q x of a diagonal QP
    rp_vec = ax - proj_S(ax, lp.lc, lp.uc)
    if row_w is not None:
        rp_vec = rp_vec * row_w
    r_p = float(np.linalg.norm(rp_vec)) / (1.0 + bnorm)
    g = lp.c - lp.ATy(y) if lp.q is None else lp.c + lp.q * x - lp.ATy(y)  # objective gradient
    xt = x - tau * g
    px = proj_X(xt, lp.lv, lp.uv)
    rd_vec = px - x
    if col_w is not None:
        rd_vec = rd_vec * col_w
    r_d = float(np.linalg.norm(rd_vec)) / tau / (1.0 + cnorm)
    s = (px - xt) / tau
    obj_p = float(np.dot(lp.c, x)) + 0.5 * quad
    obj_d = -p_fun(-y, lp.lc, lp.uc) + float(np.dot(s, x)) - 0.5 * quad
    r_g = abs(obj_p - obj_d) / (1.0 + max(abs(obj_p), abs(obj_d)))
    return dict(r_primal=r_p, r_dual=r_d, r_gap=r_g, obj_p=obj_p, obj_d=obj_d)


def p_norm_sq(dx, dy, adx, omega, eta):
    """||dz||_P^2 = (omega/eta) ||dx||^2 + (1/(eta omega)) ||dy||^2 + 2 <A dx, dy>
    (Appendix D.2.1), the metric P of Appendix B with off-diagonal blocks A^T and A."""
    return ((omega / eta) * float(np.dot(dx, dx)) + (1.0 / (eta * omega)) * float(np.dot(dy, dy))
            + 2.0 * float(np.dot(adx, dy)))


def fixed_point_residual(lp: OracleLP, x, y, xh, yh, omega, eta):
    """r(z) = ||z - PDHG(z)||_P (Appendix B.2) for z = (x, y), PDHG(z) = (x^, y^)."""
    dx = x - xh
    dy = y - yh
    return math.sqrt(max(0.0, p_norm_sq(dx, dy, lp.Ax(dx), omega, eta)))


# ----------------------------------------------------------------------------- restarts, PID
def restart_decision(r, r_anchor, r_prev, first_check, k, T, beta_s, beta_n, beta_a):
    """Restart criteria of Appendix B.2.  Returns 0 (none), 1 (sufficient decay),
    2 (necessary decay) or 3 (artificial).

    sufficient: r <= beta_s * r_anchor
    necessary:  r <= beta_n * r_anchor and r > r_prev   (not at the epoch's first check)
    artificial: k >= beta_a * T
    """
    if r <= beta_s * r_anchor:
        return 1
    if (not first_check) and r <= beta_n * r_anchor and r > r_prev:
        return 2
    if k >= beta_a * T:
        return 3
    return 0


def pid_omega(omega, d_x, d_y, e_sum, e_prev, kp, ki, kd):
    """PID primal-weight update of Appendix B.3.

    e^n = log( sqrt(omega) d_x / (d_y / sqrt(omega)) )
    log omega^{n+1} = log omega^n - [K_P e^n + K_I sum_{i<=n} e^i + K_D (e^n - e^{n-1})]

    ``e_prev`` is None at the first restart (derivative term zero).  Returns
    (omega_new, e_sum_new, e_new); skipped (omega unchanged) when d_x or d_y is zero or
    not finite."""
    if not (d_x > 0.0 and d_y > 0.0 and math.isfinite(d_x) and math.isfinite(d_y)):
        return omega, e_sum, e_prev
    so = math.sqrt(omega)
    e = math.log((so * d_x) / (d_y / so))
    e_sum = e_sum + e
    de = 0.0 if e_prev is None else (e - e_prev)
    log_w = math.log(omega) - (kp * e + ki * e_sum + kd * de)
    return math.exp(log_w), e_sum, e


def anchor_distances(xh, yh, x0, y0):
    """The PID's distances (Appendix B.3): d_x = ||x^ - x^{n,0}||, d_y = ||y^ - y^{n,0}||,
    measured from the anchor of the epoch that ends (the start point in the first epoch)."""
    return float(np.linalg.norm(xh - x0)), float(np.linalg.norm(yh - y0))


def new_epoch(S):
    """Start a restart epoch (Appendix B.2): the inner count k restarts at 0, and the
    epoch's reference r(z^{n,0}) and previous-check residual are unset until its first
    check sets both."""
    S["k"] = 0
    S["r_anchor"] = None
    S["r_prev"] = None


# ----------------------------------------------------------------------------- the solve
@dataclass
class OracleResult:
    x: np.ndarray  # x^ at the final check
    y: np.ndarray  # y^ at the final check
    status: int  # 0 converged, 1 iteration limit, 2 non-finite iterate
    iterations: int
    restarts: int
    omega: float
    eta: float
    kkt: dict
    trace: list = field(default_factory=list)
    state: dict = field(default_factory=dict)


def solve(lp: OracleLP, eps=1e-8, max_iter=100_000, params=None, x_start=None, y_start=None,
          state=None, kkt_weights=None):
    """Restarted reflected-Halpern PDHG (Algorithm 1 on one device, with Appendix B).

    Every ``check_every`` iterations, and at ``max_iter``, the check runs at the PDHG output
    (x^, y^) of that iteration: relative KKT (stop when all three are <= eps), the
    fixed-point residual, the restart test and, on restart, the PID weight update.

    ``state`` (from a previous result's ``.state``) resumes a stopped solve exactly.
    ``kkt_weights`` = (row_w, col_w, bnorm, cnorm) reports the KKT errors of another LP of
    which ``lp`` is a diagonal scaling (see ``kkt``)."""
    P = dict(DEFAULTS)
    P.update(params or {})
    n, m = lp.n, lp.m
    K = int(P["check_every"])
    row_w = col_w = None
    if kkt_weights is not None:
        row_w, col_w, bnorm, cnorm = kkt_weights
    else:
        bnorm = finite_bound_norm(lp.lc, lp.uc)
        cnorm = float(np.linalg.norm(lp.c))
    if state is not None:
        S = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in state.items()}
    else:
        eta = P["eta"] if P["eta"] is not None else default_eta(
            lp, P["eta_safety"], P["power_iters"], P["power_tol"])
        omega = P["omega0"] if P["omega0"] is not None else default_omega(lp)
        x = proj_X(np.zeros(n), lp.lv, lp.uv) if x_start is None else np.array(x_start, np.float64)
        y = np.zeros(m) if y_start is None else np.array(y_start, np.float64)
        S = dict(x=x, y=y, x0=x.copy(), y0=y.copy(), k=0, T=0, eta=float(eta), omega=float(omega),
                 r_anchor=None, r_prev=None, e_sum=0.0, e_prev=None, restarts=0, checks=0)
    x, y, x0, y0 = S["x"], S["y"], S["x0"], S["y0"]
    eta, omega = S["eta"], S["omega"]
    tau, sigma = eta / omega, eta * omega
    gamma = float(P["gamma"])
    trace = []
    status = 1
    xh = x.copy()
    yh = y.copy()
    last_kkt = {}
    while S["T"] < max_iter:
        k = S["k"]
        xh, yh, _, _ = pdhg_step(lp, x, y, tau, sigma)
        if P["halpern"]:
            xn = halpern(xh, x, x0, k, gamma)
            yn = halpern(yh, y, y0, k, gamma)
        else:
            xn, yn = xh, yh
        S["T"] += 1
        S["k"] = k + 1
        if S["T"] % K != 0 and S["T"] < max_iter:
            x, y = xn, yn
            continue
        # ---- check at the PDHG output of this iteration
        S["checks"] += 1
        last_kkt = kkt(lp, xh, yh, tau, bnorm, cnorm, row_w, col_w)
        r = fixed_point_residual(lp, x, y, xh, yh, omega, eta)
        rec = dict(T=S["T"], k=S["k"], r=r, omega=omega, restart=0, **last_kkt)
        trace.append(rec)
        if not (np.all(np.isfinite(xh)) and np.all(np.isfinite(yh)) and math.isfinite(r)):
            status = 2
            break
        if max(last_kkt["r_primal"], last_kkt["r_dual"], last_kkt["r_gap"]) <= eps:
            status = 0
            break
        first = S["r_anchor"] is None
        if first:
            S["r_anchor"] = r
            S["r_prev"] = r
        rec.update(first=first, r_anchor=S["r_anchor"], r_prev=S["r_prev"])
        kind = 0
        if P["restart"]:
            kind = restart_decision(r, S["r_anchor"], S["r_prev"], first, S["k"], S["T"],
                                    P["beta_sufficient"], P["beta_necessary"], P["beta_artificial"])
        S["r_prev"] = r
        if kind:
            rec["restart"] = kind
            S["restarts"] += 1
            if P["pid"]:
                d_x, d_y = anchor_distances(xh, yh, x0, y0)
                rec.update(d_x=d_x, d_y=d_y)
                omega, S["e_sum"], S["e_prev"] = pid_omega(
                    omega, d_x, d_y, S["e_sum"], S["e_prev"], P["pid_kp"], P["pid_ki"], P["pid_kd"])
            x0, y0 = xh.copy(), yh.copy()
            x, y = xh.copy(), yh.copy()
            new_epoch(S)
            tau, sigma = eta / omega, eta * omega
        else:
            x, y = xn, yn
    S.update(x=x, y=y, x0=x0, y0=y0, omega=omega)
    return OracleResult(x=xh, y=yh, status=status, iterations=S["T"], restarts=S["restarts"],
                        omega=omega, eta=eta, kkt=last_kkt, trace=trace, state=S)
