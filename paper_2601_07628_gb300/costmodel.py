"""Per-iteration I/O cost model of Section 3.3 (Eq. cost_model; derivation in Appendix E).

T_step(R, C) = C_spmv nnz / (B_mem N) + C_vec / B_mem (n/C + m/R)
             + C_net / B_net (n R + m C - (m + n)) / N + n_hop beta_sync (1[R>1] + 1[C>1])

with N = R C devices.  On one GPU (R = C = 1) only the two memory terms remain; they are
the paper's byte model of one PDHG iteration (24 bytes per nonzero for the CSR and CSC
passes, about 90 bytes per vector element).  ``kernel_bytes`` gives this library's own
algorithmic byte count per launch, the numerator of the roofline fractions it reports.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class CostTerms:
    spmv_s: float
    vec_s: float
    net_s: float
    latency_s: float

    @property
    def total_s(self) -> float:
        return self.spmv_s + self.vec_s + self.net_s + self.latency_s


def t_step(m: int, n: int, nnz: int, R: int = 1, C: int = 1, b_mem: float = 3350e9,
           b_net: float = 450e9, beta_sync: float = 10e-6, n_hop: int = 1, c_spmv: float = 24.0,
           c_vec: float = 90.0, c_net: float = 8.0) -> CostTerms:
    """Eq. cost_model with the parameters of Appendix E.2 as defaults (H100, FP64)."""
    N = R * C
    spmv = c_spmv * nnz / (b_mem * N)
    vec = c_vec / b_mem * (n / C + m / R)
    net = c_net / b_net * (n * R + m * C - (m + n)) / N
    lat = n_hop * beta_sync * ((1 if R > 1 else 0) + (1 if C > 1 else 0))
    return CostTerms(spmv, vec, net, lat)


def kernel_bytes(n: int, m: int, nnz: int, val_bytes: int = 8) -> dict:
    """Algorithmic HBM bytes of one launch of each fused iteration kernel.

    primal (CSC pass + primal update): nnz (value + int32 row index), n+1 int32 column
      pointers, the m-vector y gathered once, and per column 5 reads (x, x0, c, lv, uv)
      and 2 writes (x, x_bar) of 8 bytes.
    dual (CSR pass + dual update): nnz (value + int32 column index), m+1 row pointers, the
      n-vector x_bar gathered once, and per row 4 reads (y, y0, and the two bounds of -S)
      and 1 write (y).
    """
    per_nz = val_bytes + 4
    primal = per_nz * nnz + 4 * (n + 1) + 8 * m + 7 * 8 * n
    dual = per_nz * nnz + 4 * (m + 1) + 8 * n + 5 * 8 * m
    return dict(primal=primal, dual=dual, iteration=primal + dual)
