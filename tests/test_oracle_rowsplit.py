"""The all-core timing form of the oracle computes exactly the one-thread oracle.

``oracle.rowsplit.RowSplitLP`` spreads the two sparse products over host threads in
contiguous row blocks; every row keeps its stored summation order, so a solve must give
the same bits as the plain oracle, for any thread count.
"""
import numpy as np

import lpgen
from oracle import pdhg as O
from oracle.rowsplit import RowSplitLP


def test_rowsplit_products_and_solve_are_bitwise_equal():
    lp = lpgen.small_random_lp(3, n=900, m=500, nnz_per_col=6)
    base = O.OracleLP.from_lpgen(lp)
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
    ref = O.solve(base, eps=0.0, max_iter=300)
    for threads in (1, 3, 7):
        rs = RowSplitLP(base, threads)
        assert np.array_equal(rs.Ax(x), base.Ax(x)) and np.array_equal(rs.ATy(y), base.ATy(y))
        got = O.solve(rs, eps=0.0, max_iter=300)
        rs.close()
        assert np.array_equal(got.x, ref.x) and np.array_equal(got.y, ref.y), threads
        assert got.restarts == ref.restarts and got.omega == ref.omega


def test_rowsplit_handles_empty_rows_and_no_rows():
    lp = lpgen.row_length_stress_lp(5, [0, 0, 3, 0, 40, 0, 0, 1, 0], n=60)
    base = O.OracleLP.from_lpgen(lp)
    x = np.random.default_rng(1).standard_normal(lp.n)
    rs = RowSplitLP(base, 4)
    assert np.array_equal(rs.Ax(x), base.Ax(x))
    rs.close()
    box = O.OracleLP(3, 0, [1.0, -1.0, 2.0], [0], [], [], [], [], [-1.0] * 3, [1.0] * 3)
    rb = RowSplitLP(box, 2)
    assert rb.Ax(np.ones(3)).shape == (0,) and np.array_equal(rb.ATy(np.zeros(0)), np.zeros(3))
    rb.close()
