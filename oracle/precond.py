"""Diagonal preconditioning for the FP64 oracle (test infrastructure only).

The paper defines no preconditioning; its PDHG runs on the LP as given (the solver's
default).  As an option the solver scales the LP to D_r A D_c before iterating: Ruiz
equilibration in the infinity norm (each pass divides every row and column by the square
root of its largest magnitude), then one Pock-Chambolle pass with alpha = 1 (rows and
columns divided by the square root of their sums of magnitudes).  Every factor is rounded
to the nearest power of two (in the logarithm), so the scaled matrix, costs, bounds and
all conversions between scaled and original vectors are exact.

The scaled LP is  min (D_c c)^T xs  s.t.  D_r lc <= (D_r A D_c) xs <= D_r uc,
lv / D_c <= xs <= uv / D_c,  with x = D_c xs and y = D_r ys.  KKT errors are reported for
the original LP: the primal residual vector divided by D_r, the dual residual vector
(the projected step of the scaled LP) divided by D_c, the objectives unchanged.  Only
tests import this module.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import pdhg

SQRT_HALF = math.sqrt(0.5)


def pow2_nearest(v):
    """2^k with k the integer nearest to log2(v), for positive finite v (elementwise)."""
    m, e = np.frexp(np.asarray(v, np.float64))  # v = m 2^e, 0.5 <= m < 1
    return np.ldexp(1.0, np.where(m >= SQRT_HALF, e, e - 1))


def _factors(norms):
    norms = np.asarray(norms, np.float64).ravel()
    out = np.ones_like(norms)
    pos = norms > 0
    out[pos] = pow2_nearest(1.0 / np.sqrt(norms[pos]))
    return out


def scale_factors(lp: pdhg.OracleLP, ruiz_passes=10, pock_chambolle=True):
    """Row and column factors (D_r, D_c) of the preconditioner, powers of two."""
    A = abs(lp.A).tocsr().astype(np.float64)
    dr = np.ones(lp.m)
    dc = np.ones(lp.n)
    for _ in range(ruiz_passes):
        fr = _factors(A.max(axis=1).toarray()) if lp.m else np.ones(0)
        fc = _factors(A.max(axis=0).toarray()) if lp.n else np.ones(0)
        A = (sp.diags(fr) @ A @ sp.diags(fc)).tocsr()
        dr *= fr
        dc *= fc
    if pock_chambolle:
        fr = _factors(np.asarray(A.sum(axis=1))) if lp.m else np.ones(0)
        fc = _factors(np.asarray(A.sum(axis=0))) if lp.n else np.ones(0)
        dr *= fr
        dc *= fc
    return dr, dc


def scaled_lp(lp: pdhg.OracleLP, dr, dc) -> pdhg.OracleLP:
    A = (sp.diags(dr) @ lp.A @ sp.diags(dc)).tocsr()
    A.sort_indices()
    return pdhg.OracleLP(lp.n, lp.m, dc * lp.c, A.indptr, A.indices, A.data, dr * lp.lc,
                         dr * lp.uc, lp.lv / dc, lp.uv / dc,
                         None if lp.q is None else dc * dc * lp.q)


def solve(lp: pdhg.OracleLP, eps=1e-8, max_iter=100_000, params=None, x_start=None,
          y_start=None, ruiz_passes=10, pock_chambolle=True):
    """Restarted PDHG on the scaled LP; returns the oracle result with x, y in the original
    variables and KKT errors of the original LP."""
    dr, dc = scale_factors(lp, ruiz_passes, pock_chambolle)
    S = scaled_lp(lp, dr, dc)
    w = (1.0 / dr, 1.0 / dc, pdhg.finite_bound_norm(lp.lc, lp.uc), float(np.linalg.norm(lp.c)))
    res = pdhg.solve(S, eps, max_iter, params,
                     None if x_start is None else np.asarray(x_start) / dc,
                     None if y_start is None else np.asarray(y_start) / dr, kkt_weights=w)
    res.x = dc * res.x
    res.y = dr * res.y
    return res
