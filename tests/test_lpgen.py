"""The seeded workload generators match the recipes the benchmark and the tests rely on
(sizes, nonzero counts, row-length tail, value mix, row types), and their planted points
satisfy the optimality conditions they are built to satisfy (checked here with plain
numpy, independently of the oracle)."""
import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
from lpgen import EQ, LE


def csr(lp):
    return sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))


def assert_planted_optimum(lp, tol=1e-9):
    """x* feasible, y* sign-feasible, z* = c - A^T y* complementary to x*'s bounds, y* = 0 on
    rows with slack: the KKT conditions of the LP, so x* is optimal."""
    A = csr(lp)
    x, y, z = lp.x_star, lp.y_star, lp.z_star
    scale = 1.0 + np.abs(lp.b).max()
    ax = A @ x
    eq, le = lp.ctype == EQ, lp.ctype == LE
    assert np.all(np.abs(ax[eq] - lp.b[eq]) <= tol * scale)
    assert np.all(ax[le] <= lp.b[le] + tol * scale)
    assert np.all(x >= lp.lv - tol) and np.all(x <= lp.uv + tol)
    assert np.all(y[le] <= 0.0)  # '<=' rows: y <= 0 in this sign convention (y* = 0 here)
    assert np.allclose(lp.c - A.T @ y, z, atol=tol * (1.0 + np.abs(lp.c).max()))
    at_lo, at_hi = z > 0, z < 0
    assert np.all(np.abs(x[at_lo] - lp.lv[at_lo]) <= tol)
    assert np.all(np.abs(x[at_hi] - lp.uv[at_hi]) <= tol)
    slack = lp.b[le] - ax[le]
    assert np.all(np.abs(y[le][slack > tol * scale]) == 0.0)


def test_small_lp_recipe():
    lp = lpgen.small_random_lp(0)
    assert (lp.n, lp.m, lp.row_ptr[-1]) == (2000, 1000, 16000)
    A = csr(lp).tocsc()
    assert np.all(np.diff(A.indptr) == 8)  # 8 distinct rows per column
    assert int((lp.ctype == EQ).sum()) == 600 and int((lp.ctype == LE).sum()) == 400
    assert np.all(lp.lv == 0.0)
    fin = np.isfinite(lp.uv)
    assert abs(fin.mean() - 0.5) < 0.05 and np.all((lp.uv[fin] >= 1.0) & (lp.uv[fin] <= 10.0))
    assert abs(lp.val.mean()) < 0.05 and abs(lp.val.std() - 1.0) < 0.05  # N(0, 1)
    assert_planted_optimum(lp)
    # strict complementarity floor 0.1 on the bound multipliers
    assert np.all(np.abs(lp.z_star[lp.z_star != 0]) >= 0.1)


def test_powerlaw_recipe():
    """The 4M x 2M benchmark LP: 40M nonzeros within 0.1 %, Pareto row lengths capped at
    100,000 (a few dense rows), distinct columns per row, +-1 values with probability 0.7,
    60 % equality rows."""
    lp = lpgen.powerlaw_lp(1)
    assert (lp.n, lp.m) == (4_000_000, 2_000_000)
    z = int(lp.row_ptr[-1])
    assert abs(z - 40_000_000) <= 40_000 + 50_000  # bisection to 0.1 %, minus repeated draws
    L = np.diff(lp.row_ptr)
    assert L.max() <= 100_000 and L.max() >= 50_000 and L.min() >= 1
    assert 10 <= int((L >= 10_000).sum()) <= 60
    # distinct, sorted columns inside every row
    d = np.diff(lp.col.astype(np.int64))
    starts = lp.row_ptr[1:-1]
    d[starts[starts < d.shape[0] + 1] - 1] = 1  # the step across a row boundary is not checked
    assert np.all(d > 0)
    one = np.abs(lp.val) == 1.0
    assert abs(one.mean() - 0.7) < 0.01 and abs((lp.val < 0).mean() - 0.5) < 0.01
    assert abs((lp.ctype == EQ).mean() - 0.6) < 0.01
    del d, one
    assert_planted_optimum(lp, tol=1e-8)


def test_batch_recipe():
    ms = lpgen.batch_sizes(3, 256)
    assert ms.min() >= 500 and ms.max() <= 50_000 and int(ms.sum()) == 6_532_537
    for i in (0, 1):
        lp = lpgen.uneven_lp(3000 + i, int(ms[i]))
        assert lp.m == ms[i] and lp.n == 2 * lp.m
        k = np.diff(csr(lp).tocsc().indptr)
        assert k.min() >= 5 and k.max() <= 15
        assert int((lp.ctype == EQ).sum()) == (lp.m * 6) // 10
        assert_planted_optimum(lp)


def test_transport_recipe():
    fam = lpgen.transport_family(4, S=30, D=20, side_rows=200)
    lp = lpgen.transport_lp(fam, 7)
    S, D, R = 30, 20, 200
    assert lp.n == S * D and lp.m == S + D + R
    A = csr(lp)
    s, d, cap = lp.b[:S], lp.b[S:S + D], lp.b[S + D:]
    assert d.sum() == pytest.approx(0.9 * s.sum())
    # the proportional flow x_ij = s_i d_j / sum s is feasible
    x = np.outer(s, d).reshape(-1) / s.sum()
    ax = A @ x
    assert np.all(ax[:S] <= s * (1 + 1e-12))
    np.testing.assert_allclose(ax[S:S + D], d, rtol=1e-12)
    assert np.all(ax[S + D:] <= cap) and np.all(ax[S + D:] >= cap / 1.5 * (1 - 1e-12))
    assert np.all(np.diff(A.indptr)[S + D:] == 10)


def test_generators_are_seeded():
    a, b = lpgen.small_random_lp(5, n=300, m=120), lpgen.small_random_lp(5, n=300, m=120)
    assert np.array_equal(a.val, b.val) and np.array_equal(a.c, b.c)
    c = lpgen.small_random_lp(6, n=300, m=120)
    assert not np.array_equal(a.val, c.val)


# A seed names one LP on every machine: the matrix pattern, its values, the row types and
# the variable bounds come from the seeded draws alone, with no floating-point sums or
# products and no step whose order numpy leaves to the implementation (the selections
# are sorted).  The hashes below were taken on an x86 host; the same values on any other
# host (an Arm one included) show that both build the same workloads.  c and b are left
# out: they are sparse products of the planted point, which may round differently where
# a compiler contracts a multiply and an add.
def _pattern_hash(lp):
    import hashlib

    d = hashlib.sha256()
    for a, dt in ((lp.row_ptr, "<i8"), (lp.col, "<i8"), (lp.val, "<f8"), (lp.ctype, "i1"),
                  (lp.lv, "<f8"), (lp.uv, "<f8")):
        d.update(np.ascontiguousarray(np.asarray(a).astype(dt)).tobytes())
    return d.hexdigest()[:16]


_FAMILY = {}


def _transport():
    fam = _FAMILY.setdefault("t", lpgen.transport_family(4, S=20, D=20, side_rows=50))
    return lpgen.transport_lp(fam, 100)


PLATFORM_CASES = {
    "small": (lambda: lpgen.small_random_lp(0), "b8a127b948df9ec6"),
    "tiny": (lambda: lpgen.small_random_lp(7, n=250, m=125), "763535df386c07ba"),
    "stress": (lambda: lpgen.row_length_stress_lp(11, [0, 1, 33, 257, 0, 5, 1025], n=3000),
               "c833770f0c88e13a"),
    "cross": (lambda: lpgen.cross_stress_lp(5, [40, 3, 0, 33], 300, {7: 50, 11: 3}),
              "c807e565dbdcb47b"),
    "uneven": (lambda: lpgen.uneven_lp(3000, 2000), "25aa28988c0531a9"),
    "powerlaw": (lambda: lpgen.scaled_powerlaw_lp(1, 1 / 400), "7a32262c1feb2373"),
    "transport": (_transport, "9fece635b093fa80"),
    "lasso": (lambda: lpgen.lasso_qp(11, rows=300, cols=150, density=0.02, lam=0.5)[0],
              "7f99ccecd0b21e80"),
}


@pytest.mark.parametrize("case", sorted(PLATFORM_CASES))
def test_seeded_workloads_are_the_same_on_every_host(case):
    make, want = PLATFORM_CASES[case]
    assert _pattern_hash(make()) == want
