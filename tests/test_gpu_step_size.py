"""The GPU's own step size and initial primal weight against the oracle (needs a GB300).

Section 2.2 requires eta * ||A||_2 < 1 (the metric P of Appendix B is then positive
definite); the solver takes eta = 0.998 / sigma_max(A) from power iteration on A^T A and
omega_0 = ||c|| / ||b_fin|| (readings O7, O8).  The GPU runs its own power iteration (its
products in the packed kernels, its norms in its reduction kernels); here nothing is passed
in: both sides compute eta and omega_0 from the LP alone.

Tolerance: the two power iterations make the same rounds from the same start vector and
stop on the same rule; they differ only in the order of the sums inside each product and
norm (about 1e-16 relative per operation), and power iteration damps such perturbations
instead of amplifying them.  So eta agrees to about 1e-15; the bar is 1e-12.  omega_0 is
a ratio of two norms summed in different orders: same bar.
"""
import math

import numpy as np
import pytest

import lpgen
from oracle import pdhg as O
from oracle import precond as P
from parity_util import KKT_ABS, assert_xy_parity, first_divergence

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-12


@pytest.fixture(scope="session")
def Solver():
    from paper_2601_07628_gb300 import build, dpdlp

    build()
    return dpdlp.Solver


def close(a, b, tol=TOL_STEP):
    return abs(a - b) <= tol * abs(b)


def stress_lp():
    lengths = ([0, 1, 7, 31, 32, 33, 255, 256, 257, 1023, 1024, 1025, 4097, 9000, 0]
               + [5] * 300 + [17] * 100 + [1] * 400)
    return lpgen.row_length_stress_lp(12, lengths, n=20000)


def general_bounds_lp():
    lp = lpgen.small_random_lp(5, n=900, m=450, nnz_per_col=5)
    rng = np.random.default_rng(1)
    kind = rng.integers(0, 4, lp.m)
    ax = O.OracleLP.from_lpgen(lp).Ax(lp.x_star)
    lc = np.where(kind == 0, ax - 0.5, np.where(kind == 1, ax - 0.3, np.where(kind == 2, -np.inf, lp.lc)))
    uc = np.where(kind == 0, ax + 0.5, np.where(kind == 1, np.inf, np.where(kind == 2, np.inf, lp.uc)))
    return lpgen.LP(lp.n, lp.m, lp.c, lp.row_ptr, lp.col, lp.val, lc, uc, lp.lv, lp.uv, name="general")


CASES = {
    "small": lambda: lpgen.small_random_lp(0),
    "stress": stress_lp,
    "general_bounds": general_bounds_lp,
    "long_columns": lambda: lpgen.small_random_lp(4, n=40, m=12000, nnz_per_col=3000),
}


def gpu_eta_omega0(s):
    """eta of the solve and omega at its first check (the trace records omega before the
    check's PID update, so the first record holds omega_0)."""
    assert s.solve(0.0, 1) == 1
    return s.kkt()["eta"], s.trace()[0]["omega"]


@pytest.mark.parametrize("case", sorted(CASES))
def test_gpu_eta_and_omega0_match_oracle(Solver, case):
    lp = CASES[case]()
    o = O.OracleLP.from_lpgen(lp)
    eta_o, om_o = O.default_eta(o), O.default_omega(o)
    s = Solver()
    s.load(lp)
    eta_g, om_g = gpu_eta_omega0(s)
    s.close()
    assert close(eta_g, eta_o), (eta_g, eta_o)
    assert close(om_g, om_o), (om_g, om_o)


def test_gpu_eta_fixed_round_count(Solver):
    """power_tol = 0: both sides run exactly power_iters rounds (no stopping decision)."""
    lp = lpgen.small_random_lp(3, n=800, m=400, nnz_per_col=6)
    o = O.OracleLP.from_lpgen(lp)
    for rounds in (1, 7, 50):
        eta_o = O.default_eta(o, iters=rounds, tol=0.0)
        s = Solver()
        s.load(lp)
        s.set_param("power_tol", 0.0)
        s.set_param("power_iters", rounds)
        eta_g, _ = gpu_eta_omega0(s)
        s.close()
        assert close(eta_g, eta_o), (rounds, eta_g, eta_o)


def test_gpu_eta_and_omega0_preconditioned(Solver):
    """With preconditioning both are those of the scaled LP D_r A D_c (reading O15)."""
    lp = lpgen.small_random_lp(0)
    o = O.OracleLP.from_lpgen(lp)
    dr, dc = P.scale_factors(o)
    so = P.scaled_lp(o, dr, dc)
    s = Solver()
    s.set_param("precond", 1)
    s.load(lp)
    eta_g, om_g = gpu_eta_omega0(s)
    s.close()
    assert close(eta_g, O.default_eta(so)), (eta_g, O.default_eta(so))
    assert close(om_g, O.default_omega(so)), (om_g, O.default_omega(so))


def batch_lps():
    lps = [lpgen.small_random_lp(0)]
    lps += [lpgen.uneven_lp(100 + i, m) for i, m in enumerate((500, 777, 2600, 1300))]
    lps.append(lpgen.small_random_lp(4, n=300, m=120, nnz_per_col=40))
    return lps


def test_batch_eta_and_omega0_per_instance(Solver):
    """Every instance of a batch runs its own power iteration (reading O23)."""
    lps = batch_lps()
    s = Solver()
    s.load_batch(lps)
    assert s.solve(0.0, 1) == 1
    kk = s.batch_kkt()
    first = {}
    for rec in s.trace():
        first.setdefault(rec["inst"], rec["omega"])
    s.close()
    for i, lp in enumerate(lps):
        o = O.OracleLP.from_lpgen(lp)
        assert close(kk[i]["eta"], O.default_eta(o)), (i, kk[i]["eta"], O.default_eta(o))
        assert close(first[i], O.default_omega(o)), (i, first[i], O.default_omega(o))


@pytest.mark.parametrize("seed", [0, 2])
def test_free_running_with_own_step_matches_oracle(Solver, seed):
    """Nothing injected: the GPU's eta and omega_0, its own restart decisions; the oracle
    the same from the LP alone.  Same restarts, same iterates at the 1e-9 bar."""
    lp = lpgen.small_random_lp(seed, n=1500, m=700)
    o = O.OracleLP.from_lpgen(lp)
    T = 640
    ores = O.solve(o, eps=0.0, max_iter=T)
    s = Solver()
    s.load(lp)
    assert s.solve(0.0, T) == 1
    x, y = s.solution()
    tr = s.trace()
    k = s.kkt()
    s.close()
    rep = first_divergence(tr, ores.trace)  # the first differing decision, if any
    assert rep is None, rep
    assert close(k["eta"], ores.eta)
    assert abs(k["omega"] - ores.omega) <= 1e-9 * ores.omega
    assert_xy_parity(x, y, ores.x, ores.y, 1e-9)
    for key in ("r_primal", "r_dual", "r_gap"):
        assert math.isclose(k[key], ores.kkt[key], rel_tol=1e-6, abs_tol=KKT_ABS), key
