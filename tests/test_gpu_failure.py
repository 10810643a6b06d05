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
