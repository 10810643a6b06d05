"""Failure detection on the GPU, injected on the host, with no GPU fault.

A step size far above the stability bound eta < 1 / ||A|| (eta = 1e300) makes the iterates
overflow to inf and NaN.  Then:
* the check must report DPDLP_NUMERICAL (2) at the first check, as the oracle does;
* the handle must stay usable for the next solve;
* in a batch the failure must stay with its instance: the others still converge, and the
  batch status is the worst instance status.
"""
import numpy as np
import pytest

import lpgen
from oracle import pdhg as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def Solver():
    from paper_2601_07628_gb300 import build, dpdlp

    build()
    return dpdlp.Solver


def test_nonfinite_iterates_are_reported(Solver):
    lp = lpgen.small_random_lp(0, n=200, m=100)
    with np.errstate(all="ignore"):
        ref = O.solve(O.OracleLP.from_lpgen(lp), eps=1e-8, max_iter=640, params=dict(eta=1e300))
    assert ref.status == 2
    s = Solver()
    s.load(lp)
    s.set_param("eta", 1e300)
    assert s.solve(1e-8, 640) == 2
    k = s.kkt()
    assert k["status"] == 2 and k["iterations"] == ref.iterations
    s.set_param("eta", 0.0)  # back to the power-iteration step: the handle still works
    assert s.solve(1e-6, 200_000) == 0
    s.close()


def test_batch_isolates_a_diverging_instance(Solver):
    lps = [lpgen.small_random_lp(0, n=200, m=100), lpgen.small_random_lp(1, n=300, m=150)]
    solo = Solver()
    solo.load(lps[0])
    assert solo.solve(1e-6, 200_000) == 0
    want = solo.kkt()
    solo.close()
    s = Solver()
    s.load_batch(lps)
    s.solve(1e-6, 64)
    eta0 = s.batch_kkt()[0]["eta"]
    s.set_batch_eta([eta0, 1e300])
    assert s.solve(1e-6, 200_000) == 2  # the worst instance status
    kk = s.batch_kkt()
    assert kk[1]["status"] == 2 and kk[1]["iterations"] == 64
    assert kk[0]["status"] == 0 and kk[0]["iterations"] == want["iterations"]
    assert kk[0]["eta"] == want["eta"]
    s.close()


def test_batch_isolates_a_diverging_first_instance(Solver):
    """The first instance owns entry 0 of the stacked vectors, the entry that padding and
    the stored zero of an empty row gather in a single LP (0 times that entry).  With the
    first instance diverging, an instance with empty rows and empty columns still
    converges as it does alone: its own stored zeros gather its own first entry."""
    other = lpgen.row_length_stress_lp(12, [0, 5, 9, 0, 17, 3] * 40 + [0], n=400)
    assert (np.diff(other.row_ptr) == 0).sum() > 0
    assert (np.bincount(other.col, minlength=other.n) == 0).sum() > 0
    solo = Solver()
    solo.set_param("perm_seed", 1 + 2 * 1)  # the block permutation of instance 1 in a batch
    solo.load(other)
    assert solo.solve(1e-6, 200_000) == 0
    want = solo.kkt()
    want_xy = solo.solution()
    solo.close()
    s = Solver()
    s.load_batch([lpgen.small_random_lp(0, n=200, m=100), other])
    s.solve(1e-6, 64)
    eta1 = s.batch_kkt()[1]["eta"]
    s.set_batch_eta([1e300, eta1])
    assert s.solve(1e-6, 200_000) == 2
    kk = s.batch_kkt()
    assert kk[0]["status"] == 2 and kk[0]["iterations"] == 64
    assert kk[1]["status"] == 0 and kk[1]["iterations"] == want["iterations"]
    assert kk[1]["eta"] == want["eta"]
    x1, y1 = s.split(*s.solution())[1]
    assert np.array_equal(x1, want_xy[0]) and np.array_equal(y1, want_xy[1])
    s.close()
