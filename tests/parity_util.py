"""Vector comparisons shared by the GPU parity tests (no oracle arithmetic here).

The parity bar compares the GPU's iterates with the oracle's two ways:
* relative 2-norm: ||g - r|| / ||r|| <= tol, the bar of the whole vector;
* element by element: max_i |g_i - r_i| <= tol * max(||r||_inf, 1), so that a few wrong
  entries (one bad row of a slot, one long row) cannot hide inside a 2-norm over millions.
"""
import numpy as np

# KKT values (relative residuals and gap) are compared at 1e-6 relative, or within KKT_ABS
# absolutely.  The gap |obj_p - obj_d| / (1 + max |obj|) is a difference of two objectives,
# each a sum of n (or m) products that the two sides add in different orders: each sum is
# off by up to about n u sum|terms| (u = 1.1e-16), which at these sizes (n up to a few
# thousand, sum|terms| a few times |obj|) is 1e-13 to 1e-12 of 1 + max |obj|.  Once the
# gap itself is near 1e-8 that rounding is all that separates the two sides, so the
# relative bar alone would demand more than FP64 gives; the residual norms are bounded the
# same way.
KKT_ABS = 1e-12


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def max_elem_err(a, b):
    """max_i |a_i - b_i| / max(||b||_inf, 1)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if b.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1.0))


def vec_errors(a, b):
    return rel(a, b) if np.asarray(b).size else 0.0, max_elem_err(a, b)


def assert_vec_parity(a, b, tol, what=""):
    e2, ei = vec_errors(a, b)
    assert e2 <= tol and ei <= tol, (what, e2, ei)


def assert_xy_parity(x, y, xr, yr, tol, what=""):
    assert_vec_parity(x, xr, tol, f"{what} x")
    assert_vec_parity(y, yr, tol, f"{what} y")


def first_divergence(gpu_trace, oracle_trace):
    """Parity report of free-running solves (reading O21): the first check at which the GPU's
    and the oracle's restart decisions (or check iterations) differ, as a dict with the
    check index, both records' iteration, decision and KKT values, or None when both traces
    agree and have the same length.  GPU records name the fixed-point residual r_fp, the
    oracle's r."""
    keys = ("T", "restart", "r_primal", "r_dual", "r_gap")
    for i, (g, o) in enumerate(zip(gpu_trace, oracle_trace)):
        if g["restart"] != o["restart"] or g["T"] != o["T"]:
            return {"check": i, "gpu": {k: g[k] for k in keys}, "oracle": {k: o[k] for k in keys}}
    if len(gpu_trace) != len(oracle_trace):
        return {"check": min(len(gpu_trace), len(oracle_trace)), "gpu_checks": len(gpu_trace),
                "oracle_checks": len(oracle_trace)}
    return None
