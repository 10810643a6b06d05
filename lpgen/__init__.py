"""Seeded synthetic LP generators shared by the tests, the benchmark and the oracle checks.

This module builds problem data only.  It holds none of the solver's arithmetic: no PDHG
step, no projection, no residual.  Every LP it returns is in the form of Section 2.1
(Eq. prob:primal): ``min c^T x  s.t.  lc <= A x <= uc,  lv <= x <= uv`` with ``A`` stored
as CSR (int64 row pointers, int32 column indices sorted inside each row, float64 values).

Row types follow the constraint-type codes of the C ABI: 0 is an equality row
(``lc = uc = b``), 1 a ``<=`` row (``lc = -inf, uc = b``), 2 a ``>=`` row
(``lc = b, uc = +inf``).

Feasible instances are built from a primal-dual pair ``(x*, y*, z*)`` that satisfies the
KKT conditions of the LP by construction, so the optimal value ``p* = c^T x*`` is known
without solving anything:

* ``x*`` sits at its lower bound, its upper bound, or strictly inside;
* ``<=`` rows get a positive slack and ``y* = 0``; equality rows get ``y* ~ N(0, 1)``;
* the reduced cost ``z*`` is positive at a lower bound, negative at an upper bound and
  zero inside (strict complementarity, with a 0.1 floor);
* ``c = A^T y* + z*``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

EQ, LE, GE = 0, 1, 2


@dataclasses.dataclass
class LP:
    """A sparse LP in CSR form, plus the optimal pair it was built from (if any)."""

    n: int
    m: int
    c: np.ndarray
    row_ptr: np.ndarray  # int64 [m+1]
    col: np.ndarray  # int32 [Z]
    val: np.ndarray  # float64 [Z]
    lc: np.ndarray  # float64 [m], -inf allowed
    uc: np.ndarray  # float64 [m], +inf allowed
    lv: np.ndarray  # float64 [n], -inf allowed
    uv: np.ndarray  # float64 [n], +inf allowed
    ctype: np.ndarray | None = None  # int8 [m] when every row is one of EQ/LE/GE
    b: np.ndarray | None = None  # float64 [m], the finite side of each typed row
    x_star: np.ndarray | None = None
    y_star: np.ndarray | None = None
    z_star: np.ndarray | None = None
    name: str = "lp"
    q: np.ndarray | None = None  # float64 [n] >= 0: diagonal QP objective 1/2 x^T diag(q) x + c^T x

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def p_star(self) -> float | None:
        if self.x_star is None:
            return None
        return float(np.dot(self.c, self.x_star))


def bounds_from_types(ctype: np.ndarray, b: np.ndarray):
    """Row bounds (lc, uc) from constraint-type codes and right-hand sides."""
    lc = np.where(ctype == LE, -np.inf, b).astype(np.float64)
    uc = np.where(ctype == GE, np.inf, b).astype(np.float64)
    return lc, uc


def _csr_from_coo(m: int, n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray):
    """CSR arrays with columns sorted inside each row; (row, col) pairs must be distinct."""
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order]
    vals = vals[order]
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), vals.astype(np.float64)


def _csr_matvec(row_ptr, col, val, x):
    """A x for building right-hand sides (construction only, not solver arithmetic)."""
    m = row_ptr.shape[0] - 1
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    return np.bincount(rows, weights=val * x[col], minlength=m)


def _csr_rmatvec(row_ptr, col, val, y, n):
    m = row_ptr.shape[0] - 1
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    return np.bincount(col, weights=val * y[rows], minlength=n)


def _planted_optimum(rng, n, m, row_ptr, col, val, ctype):
    """Bounds, x*, y*, z*, b and c for a feasible LP with a known optimum."""
    lv = np.zeros(n)
    uv = np.full(n, np.inf)
    finite_u = rng.random(n) < 0.5
    uv[finite_u] = rng.uniform(1.0, 10.0, size=int(finite_u.sum()))
    # Category per variable: 0 at lower bound, 1 at upper bound, 2 interior.
    # Finite-u variables: 40 % lower / 40 % upper / 20 % inside; the others 40 % / 0 / 60 %,
    # so over all variables 40 % sit at 0 and 20 % at u.
    r = rng.random(n)
    cat = np.where(r < 0.4, 0, np.where(finite_u & (r < 0.8), 1, 2))
    x_star = np.zeros(n)
    x_star[cat == 1] = uv[cat == 1]
    inside = cat == 2
    hi = np.where(np.isfinite(uv), uv, 10.0)
    x_star[inside] = rng.uniform(0.0, 1.0, size=int(inside.sum())) * hi[inside]
    z_star = np.zeros(n)
    z_star[cat == 0] = rng.uniform(0.1, 1.0, size=int((cat == 0).sum()))
    z_star[cat == 1] = -rng.uniform(0.1, 1.0, size=int((cat == 1).sum()))
    ax = _csr_matvec(row_ptr, col, val, x_star)
    b = np.array(ax, dtype=np.float64)
    le = ctype == LE
    b[le] += rng.uniform(0.0, 1.0, size=int(le.sum()))
    y_star = np.zeros(m)
    eq = ctype == EQ
    y_star[eq] = rng.standard_normal(int(eq.sum()))
    c = _csr_rmatvec(row_ptr, col, val, y_star, n) + z_star
    return lv, uv, x_star, y_star, z_star, b, c


def small_random_lp(seed: int = 0, n: int = 2000, m: int = 1000, nnz_per_col: int = 8,
                    n_eq: int | None = None) -> LP:
    """Small feasible LP: every column holds ``nnz_per_col`` distinct rows drawn uniformly,
    values N(0, 1); the first 60 % of rows are equalities and the rest ``<=`` rows.

    With the defaults this is the 2,000-variable, 1,000-row workload (600 equality rows,
    400 ``<=`` rows, 16,000 nonzeros).
    """
    rng = np.random.default_rng(seed)
    if n_eq is None:
        n_eq = (m * 6) // 10
    k = min(nnz_per_col, m)
    # the k rows of smallest key per column, in increasing row order: argpartition leaves
    # the order of the selected entries to the implementation (it differs between numpy's
    # SIMD and generic selection), and the values below are assigned in this order
    rows = np.sort(np.argpartition(rng.random((n, m)), k - 1, axis=1)[:, :k], axis=1).reshape(-1) \
        if m > 0 else np.zeros(0, dtype=np.int64)
    cols = np.repeat(np.arange(n), k) if m > 0 else np.zeros(0, dtype=np.int64)
    vals = rng.standard_normal(rows.shape[0])
    row_ptr, col, val = _csr_from_coo(m, n, rows.astype(np.int64), cols.astype(np.int64), vals)
    ctype = np.where(np.arange(m) < n_eq, EQ, LE).astype(np.int8)
    lv, uv, xs, ys, zs, b, c = _planted_optimum(rng, n, m, row_ptr, col, val, ctype)
    lc, uc = bounds_from_types(ctype, b)
    return LP(n, m, c, row_ptr, col, val, lc, uc, lv, uv, ctype, b, xs, ys, zs,
              name=f"small_random_lp(seed={seed},n={n},m={m})")


def _pareto_row_lengths(rng, m: int, target_nnz: int, cap: int, alpha: float = 1.5):
    """Row lengths L_i = min(cap, ceil(L0 * U^(-1/alpha))) with L0 chosen by bisection so
    that sum(L) is within 0.1 % of ``target_nnz`` (Pareto tail of index ``alpha``)."""
    u = 1.0 - rng.random(m)  # in (0, 1]
    base = u ** (-1.0 / alpha)

    def total(l0):
        return int(np.minimum(cap, np.ceil(l0 * base)).sum())

    lo, hi = 1e-3, float(target_nnz) / m * 4 + 1.0
    while total(hi) < target_nnz and hi < 1e9:
        hi *= 2
    l0 = hi
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        t = total(mid)
        if abs(t - target_nnz) <= max(1, target_nnz // 1000):
            l0 = mid
            break
        if t < target_nnz:
            lo = mid
        else:
            hi = mid
            l0 = mid
    lengths = np.minimum(cap, np.ceil(l0 * base)).astype(np.int64)
    return lengths, l0


def powerlaw_lp(seed: int = 1, n: int = 4_000_000, m: int = 2_000_000,
                target_nnz: int = 40_000_000, cap: int = 100_000, eq_frac: float = 0.6,
                alpha: float = 1.5) -> LP:
    """Large irregular LP with power-law row lengths.

    Row lengths follow a Pareto tail of index 1.5 capped at ``cap`` (a few rows are dense and
    stress load balance); each row picks distinct columns uniformly at random; values are
    +-1 with probability 0.7 and +-lognormal(0, 1) otherwise; ``eq_frac`` of the rows
    (chosen at random) are equalities and the others ``<=`` rows; bounds and the planted
    optimum are built as in :func:`small_random_lp`.

    With the defaults this is the 4M-variable, 2M-row, ~40M-nonzero workload.
    """
    rng = np.random.default_rng(seed)
    cap = min(cap, n)
    lengths, _ = _pareto_row_lengths(rng, m, target_nnz, cap, alpha)
    rows = np.repeat(np.arange(m, dtype=np.int64), lengths)
    cols = rng.integers(0, n, size=rows.shape[0], dtype=np.int64)
    key = rows * n + cols
    del rows, cols
    key.sort()  # by (row, col); then drop repeated draws inside a row
    keep = np.empty(key.shape[0], dtype=bool)
    keep[:1] = True
    np.not_equal(key[1:], key[:-1], out=keep[1:])
    key = key[keep]
    del keep
    rows = key // n
    cols = (key - rows * n).astype(np.int32)
    del key
    z = rows.shape[0]
    mag = np.where(rng.random(z) < 0.7, 1.0, rng.lognormal(0.0, 1.0, size=z))
    vals = np.where(rng.random(z) < 0.5, -mag, mag)
    del mag
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    del rows
    ctype = np.where(rng.random(m) < eq_frac, EQ, LE).astype(np.int8)
    lv, uv, xs, ys, zs, b, c = _planted_optimum(rng, n, m, row_ptr, cols, vals, ctype)
    lc, uc = bounds_from_types(ctype, b)
    return LP(n, m, c, row_ptr, cols, vals, lc, uc, lv, uv, ctype, b, xs, ys, zs,
              name=f"powerlaw_lp(seed={seed},n={n},m={m},nnz~{target_nnz})")


def tiny_bounded_lp(seed: int, n: int = 4, m: int = 3, density: float = 0.7) -> LP:
    """Tiny dense-ish LP with finite variable bounds (a polytope), mixed row types and an
    interior feasible point, for brute-force vertex enumeration."""
    rng = np.random.default_rng(seed)
    dense = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
    for i in range(m):  # no empty rows
        if not dense[i].any():
            dense[i, rng.integers(n)] = rng.standard_normal() or 1.0
    lv = -rng.uniform(0.0, 2.0, size=n)
    uv = rng.uniform(0.5, 3.0, size=n)
    xf = lv + (uv - lv) * rng.uniform(0.2, 0.8, size=n)
    ax = dense @ xf
    ctype = rng.integers(0, 3, size=m).astype(np.int8)
    slack = rng.uniform(0.1, 1.0, size=m)
    b = np.where(ctype == EQ, ax, np.where(ctype == LE, ax + slack, ax - slack))
    lc, uc = bounds_from_types(ctype, b)
    c = rng.standard_normal(n)
    rr, cc = np.nonzero(dense)
    row_ptr, col, val = _csr_from_coo(m, n, rr.astype(np.int64), cc.astype(np.int64), dense[rr, cc])
    return LP(n, m, c, row_ptr, col, val, lc, uc, lv, uv, ctype, b, name=f"tiny_bounded_lp({seed})")


def from_dense(A: np.ndarray, c, lc, uc, lv, uv, name="dense") -> LP:
    """Wrap a small dense matrix as an LP in CSR form (structural zeros dropped)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    rr, cc = np.nonzero(A)
    row_ptr, col, val = _csr_from_coo(m, n, rr.astype(np.int64), cc.astype(np.int64), A[rr, cc])
    f = lambda v, k: np.asarray(v, dtype=np.float64).reshape(k)
    return LP(n, m, f(c, n), row_ptr, col, val, f(lc, m), f(uc, m), f(lv, n), f(uv, n), name=name)


def row_length_stress_lp(seed: int, lengths, n: int) -> LP:
    """LP whose rows have exactly the given lengths (distinct uniform columns, N(0,1) values),
    mixed row types and a planted optimum: used to stress SpMV load balancing (empty rows,
    single long rows, rows that straddle tile boundaries)."""
    rng = np.random.default_rng(seed)
    lengths = np.asarray(lengths, dtype=np.int64)
    m = lengths.shape[0]
    rows_l, cols_l = [], []
    for i, L in enumerate(lengths):
        if L == 0:
            continue
        L = int(min(L, n))
        cols_l.append(rng.choice(n, size=L, replace=False))
        rows_l.append(np.full(L, i, dtype=np.int64))
    rows = np.concatenate(rows_l) if rows_l else np.zeros(0, np.int64)
    cols = np.concatenate(cols_l).astype(np.int64) if cols_l else np.zeros(0, np.int64)
    vals = rng.standard_normal(rows.shape[0])
    row_ptr, col, val = _csr_from_coo(m, n, rows, cols, vals)
    ctype = rng.integers(0, 3, size=m).astype(np.int8)
    ctype[ctype == GE] = LE  # planted optimum uses EQ / LE rows
    lv, uv, xs, ys, zs, b, c = _planted_optimum(rng, n, m, row_ptr, col, val, ctype)
    lc, uc = bounds_from_types(ctype, b)
    return LP(n, m, c, row_ptr, col, val, lc, uc, lv, uv, ctype, b, xs, ys, zs,
              name=f"row_length_stress_lp({seed})")


def cross_stress_lp(seed: int, lengths, n: int, dense_cols: dict) -> LP:
    """LP whose rows have the given lengths (distinct uniform columns, as
    ``row_length_stress_lp``) and whose columns ``j`` in ``dense_cols`` additionally hold
    ``dense_cols[j]`` distinct uniform rows, so both A and A^T have rows of chosen lengths;
    N(0,1) values, '=' / '<=' rows and a planted optimum."""
    rng = np.random.default_rng(seed)
    lengths = np.asarray(lengths, dtype=np.int64)
    m = lengths.shape[0]
    pairs = set()
    for i, L in enumerate(lengths):
        for j in rng.choice(n, size=int(min(L, n)), replace=False):
            pairs.add((i, int(j)))
    for j, k in dense_cols.items():
        for i in rng.choice(m, size=int(min(k, m)), replace=False):
            pairs.add((int(i), int(j)))
    pr = np.array(sorted(pairs), dtype=np.int64).reshape(-1, 2)
    vals = rng.standard_normal(pr.shape[0])
    row_ptr, col, val = _csr_from_coo(m, n, pr[:, 0], pr[:, 1], vals)
    ctype = rng.integers(0, 2, size=m).astype(np.int8)  # EQ / LE rows
    lv, uv, xs, ys, zs, b, c = _planted_optimum(rng, n, m, row_ptr, col, val, ctype)
    lc, uc = bounds_from_types(ctype, b)
    return LP(n, m, c, row_ptr, col, val, lc, uc, lv, uv, ctype, b, xs, ys, zs,
              name=f"cross_stress_lp({seed})")


def scaled_powerlaw_lp(seed: int, scale: float) -> LP:
    """The power-law workload shrunk by ``scale`` in n, m and nnz (same recipe, cap scaled)."""
    n = max(2, int(round(4_000_000 * scale)))
    m = max(1, int(round(2_000_000 * scale)))
    z = max(m, int(round(40_000_000 * scale)))
    cap = max(1, min(n, int(round(100_000 * math.sqrt(scale)))))
    return powerlaw_lp(seed=seed, n=n, m=m, target_nnz=z, cap=cap)


def _distinct_rows_per_column(rng, m: int, k: np.ndarray, draws: int = 24) -> np.ndarray:
    """For column j, k[j] distinct rows uniformly at random (rows in draw order; a
    sequential draw without replacement).  Returns the rows, column-major."""
    n = k.shape[0]
    kmax = int(k.max()) if n else 0
    if n == 0 or m == 0:
        return np.zeros(0, dtype=np.int64)
    cand = rng.integers(0, m, size=(n, max(draws, kmax)))
    order = np.argsort(cand, axis=1, kind="stable")
    srt = np.take_along_axis(cand, order, 1)
    first = np.ones(srt.shape, dtype=bool)
    first[:, 1:] = srt[:, 1:] != srt[:, :-1]
    keep = np.zeros(srt.shape, dtype=bool)
    np.put_along_axis(keep, order, first, 1)  # first occurrence of each row, draw order
    rank = np.cumsum(keep, axis=1) - 1
    sel = keep & (rank < k[:, None])
    short = np.nonzero(sel.sum(axis=1) < k)[0]
    rows = [cand[j][sel[j]] for j in range(n)] if short.size else None
    if rows is None:
        return cand[sel]
    for j in short:  # rare: too few distinct draws, take a fresh subset
        rows[j] = rng.choice(m, size=int(k[j]), replace=False)
    return np.concatenate(rows)


def uneven_lp(seed: int, m: int, n: int | None = None, nnz_lo: int = 5, nnz_hi: int = 15) -> LP:
    """One instance of the batched workload: ``n = 2 m`` columns by default, each holding
    U{nnz_lo..nnz_hi} distinct rows drawn uniformly, values N(0, 1); the first 60 % of rows
    are equalities and the rest ``<=`` rows; bounds and planted optimum as
    ``small_random_lp``."""
    rng = np.random.default_rng(seed)
    n = 2 * m if n is None else n
    k = np.minimum(rng.integers(nnz_lo, nnz_hi + 1, size=n), m)
    rows = _distinct_rows_per_column(rng, m, k)
    cols = np.repeat(np.arange(n, dtype=np.int64), k)
    vals = rng.standard_normal(rows.shape[0])
    row_ptr, col, val = _csr_from_coo(m, n, rows.astype(np.int64), cols, vals)
    ctype = np.where(np.arange(m) < (m * 6) // 10, EQ, LE).astype(np.int8)
    lv, uv, xs, ys, zs, b, c = _planted_optimum(rng, n, m, row_ptr, col, val, ctype)
    lc, uc = bounds_from_types(ctype, b)
    return LP(n, m, c, row_ptr, col, val, lc, uc, lv, uv, ctype, b, xs, ys, zs,
              name=f"uneven_lp(seed={seed},m={m},n={n})")


def batch_sizes(seed: int = 3, count: int = 256, m_lo: int = 500, m_hi: int = 50_000) -> np.ndarray:
    """Row counts m_i ~ U{m_lo..m_hi} of the batched workload."""
    return np.random.default_rng(seed).integers(m_lo, m_hi + 1, size=count)


def batch_lps(seed: int = 3, count: int = 256, m_lo: int = 500, m_hi: int = 50_000) -> list:
    """The batched workload: ``count`` independent LPs of uneven sizes (m_i ~ U{m_lo..m_hi},
    n_i = 2 m_i, 5-15 nonzeros per column).  Instance i is ``uneven_lp`` with seed
    1000 * seed + i.  With the defaults: 256 LPs, about 6.5M rows, 12.9M columns and 129M
    nonzeros in total."""
    ms = batch_sizes(seed, count, m_lo, m_hi)
    return [uneven_lp(1000 * seed + i, int(mi)) for i, mi in enumerate(ms)]


# ---------------------------------------------------------------- transportation family
def transport_family(seed: int = 4, S: int = 300, D: int = 300, side_rows: int = 20_000,
                     arcs_per_side: int = 10) -> dict:
    """Shared structure of a family of transportation LPs (one matrix, perturbed b and c).

    Arc (i, j) from source i to sink j is variable i * D + j, x >= 0.  Rows: S supply rows
    sum_j x_ij <= s_i, D demand rows sum_i x_ij = d_j, and ``side_rows`` capacity rows, each
    over ``arcs_per_side`` distinct random arcs.  Returns the base costs U(1, 100), the base
    supplies and demands, and the side rows' arc lists."""
    rng = np.random.default_rng(seed)
    n = S * D
    side = np.stack([rng.choice(n, size=arcs_per_side, replace=False) for _ in range(side_rows)]) \
        if side_rows else np.zeros((0, arcs_per_side), np.int64)
    return dict(S=S, D=D, n=n, side=side.astype(np.int64),
                c_base=rng.uniform(1.0, 100.0, size=n),
                s_base=rng.uniform(50.0, 150.0, size=S),
                d_base=rng.uniform(50.0, 150.0, size=D))


def transport_lp(fam: dict, seed: int) -> LP:
    """One instance of a transportation family: costs c_base * U(0.9, 1.1) per arc, supplies
    and demands s_base, d_base * U(0.8, 1.2), demands scaled so sum d = 0.9 sum s, and side
    capacities cap_r = (1 + U(0, 0.5)) * sum_{arcs in r} s_i d_j / sum s, so the proportional
    flow x_ij = s_i d_j / sum s is feasible.  The optimum is not planted (x_star etc. are
    None)."""
    rng = np.random.default_rng(seed)
    S, D, n, side = fam["S"], fam["D"], fam["n"], fam["side"]
    c = fam["c_base"] * rng.uniform(0.9, 1.1, size=n)
    s = fam["s_base"] * rng.uniform(0.8, 1.2, size=S)
    d = fam["d_base"] * rng.uniform(0.8, 1.2, size=D)
    d *= 0.9 * s.sum() / d.sum()
    src, snk = side // D, side % D
    cap = (1.0 + rng.uniform(0.0, 0.5, size=side.shape[0])) * (s[src] * d[snk]).sum(axis=1) / s.sum()
    R = side.shape[0]
    if "_shared" not in fam:  # the matrix, row types and bounds are the family's, built once
        m = S + D + R
        rows = np.concatenate([np.repeat(np.arange(S), D),                       # supply rows
                               S + np.tile(np.arange(D), S),                     # demand rows
                               S + D + np.repeat(np.arange(R), side.shape[1])])  # side rows
        cols = np.concatenate([np.arange(n), np.arange(n), side.reshape(-1)])
        vals = np.ones(rows.shape[0])
        row_ptr, col, val = _csr_from_coo(m, n, rows.astype(np.int64), cols.astype(np.int64), vals)
        ctype = np.concatenate([np.full(S, LE), np.full(D, EQ), np.full(R, LE)]).astype(np.int8)
        fam["_shared"] = (m, row_ptr, col, val, ctype, np.zeros(n), np.full(n, np.inf))
    m, row_ptr, col, val, ctype, lv, uv = fam["_shared"]
    b = np.concatenate([s, d, cap])
    lc, uc = bounds_from_types(ctype, b)
    return LP(n, m, c, row_ptr, col, val, lc, uc, lv, uv, ctype, b, None, None, None,
              name=f"transport_lp(S={S},D={D},R={R},seed={seed})")


# ---------------------------------------------------------------- diagonal QP (LASSO)
def lasso_qp(seed: int, rows: int, cols: int, density: float = 0.1, lam: float = 0.1):
    """LASSO min 1/2 ||M x - d||^2 + lam ||x||_1 written as a diagonal QP over (x, r, t):
    min 1/2 r^T r + lam 1^T t  s.t.  M x - r = d,  x - t <= 0,  x + t >= 0,  t >= 0
    (Q = I on r, 0 elsewhere).  M is sparse N(0,1), round(density * rows) distinct uniform
    rows per column, d = M x_true + noise
    for a sparse x_true.  Returns (LP with q set, {"M" (CSR), "d", "lam", "x": indices of x})."""
    rng = np.random.default_rng(seed)
    k = np.full(cols, max(1, int(round(density * rows))))  # nonzeros per column of M
    ri = _distinct_rows_per_column(rng, rows, k)
    ci = np.repeat(np.arange(cols), k)
    Msp = sp.csr_matrix((rng.standard_normal(ri.shape[0]), (ri, ci)), shape=(rows, cols))
    Msp.sort_indices()
    xt = np.where(rng.random(cols) < 0.2, rng.standard_normal(cols), 0.0)
    d = Msp @ xt + 0.1 * rng.standard_normal(rows)
    I_c, I_r = sp.identity(cols, format="csr"), sp.identity(rows, format="csr")
    Z_rc = sp.csr_matrix((rows, cols))
    Z_cr = sp.csr_matrix((cols, rows))
    A = sp.vstack([sp.hstack([Msp, -I_r, Z_rc]),      # M x - r = d
                   sp.hstack([I_c, Z_cr, -I_c]),      # x - t <= 0
                   sp.hstack([I_c, Z_cr, I_c])]).tocsr()  # x + t >= 0
    A.sort_indices()
    n = 2 * cols + rows
    m = rows + 2 * cols
    ctype = np.concatenate([np.full(rows, EQ), np.full(cols, LE), np.full(cols, GE)]).astype(np.int8)
    b = np.concatenate([d, np.zeros(2 * cols)])
    c = np.concatenate([np.zeros(cols + rows), np.full(cols, lam)])
    q = np.concatenate([np.zeros(cols), np.ones(rows), np.zeros(cols)])
    lv = np.concatenate([np.full(cols + rows, -np.inf), np.zeros(cols)])
    uv = np.full(n, np.inf)
    lc, uc = bounds_from_types(ctype, b)
    lp = LP(n, m, c, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64),
            lc, uc, lv, uv, ctype, b, name=f"lasso_qp(seed={seed},rows={rows},cols={cols})", q=q)
    return lp, {"M": Msp, "d": d, "lam": lam, "x": np.arange(cols)}
