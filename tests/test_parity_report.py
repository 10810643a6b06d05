"""The parity report of free-running solves (``parity_util.first_divergence``), on the CPU:
it names the first check whose restart decision or iteration differs, and nothing when the
traces agree.  The oracle's own traces serve as both sides here."""
import copy

import lpgen
from oracle import pdhg as O
from parity_util import first_divergence


def _trace():
    lp = lpgen.small_random_lp(3, n=300, m=150)
    return O.solve(O.OracleLP.from_lpgen(lp), eps=0.0, max_iter=640).trace


def test_agreeing_traces_report_nothing():
    t = _trace()
    assert first_divergence(copy.deepcopy(t), t) is None


def test_first_differing_decision_is_reported():
    t = _trace()
    g = copy.deepcopy(t)
    i = next(k for k, r in enumerate(t) if r["restart"] == 0 and k > 0)
    g[i]["restart"] = 2
    g[i + 1]["restart"] = 3  # a later difference is not the first
    rep = first_divergence(g, t)
    assert rep["check"] == i and rep["gpu"]["restart"] == 2 and rep["oracle"]["restart"] == 0
    assert rep["gpu"]["T"] == rep["oracle"]["T"] == t[i]["T"]
    assert rep["oracle"]["r_gap"] == t[i]["r_gap"]


def test_shifted_check_and_length_are_reported():
    t = _trace()
    g = copy.deepcopy(t)
    g[4]["T"] += 1
    assert first_divergence(g, t)["check"] == 4
    rep = first_divergence(copy.deepcopy(t[:-2]), t)
    assert rep == {"check": len(t) - 2, "gpu_checks": len(t) - 2, "oracle_checks": len(t)}
