"""The FP64 oracle with its sparse products spread over host threads (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and by the CPU legs of ``bench.py`` (the
oracle timed on all host cores); the product path never uses it.

``RowSplitLP`` is an ``OracleLP`` whose two products, A x and A^T y, are computed as
contiguous row blocks, one block per thread.  Each row is still summed left to right in
stored order by scipy's CSR kernel (which releases the interpreter lock), and every row is
written by exactly one thread, so the products -- and with them every iterate of
``pdhg.solve`` -- are bitwise those of the one-thread oracle.  Nothing else changes: the
vector updates, norms and dots stay in numpy on the calling thread.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .pdhg import OracleLP


def _blocks(M, parts):
    """Contiguous row blocks of CSR matrix M with about equal nonzero counts."""
    rows = M.shape[0]
    if rows == 0:
        return [(0, 0, M)]
    targets = np.linspace(0, M.nnz, parts + 1)
    cuts = np.searchsorted(M.indptr, targets[1:-1], side="left")
    bounds = np.unique(np.concatenate([[0], np.clip(cuts, 0, rows), [rows]]))
    return [(int(a), int(b), M[int(a):int(b)]) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]


class RowSplitLP(OracleLP):
    """The LP of ``base`` with A x and A^T y computed by ``threads`` host threads."""

    def __init__(self, base: OracleLP, threads: int | None = None):
        self.__dict__.update(base.__dict__)
        self.threads = int(threads or os.cpu_count() or 1)
        self._pool = ThreadPoolExecutor(self.threads) if self.threads > 1 else None
        self._A_blocks = _blocks(self.A, self.threads)
        self._AT_blocks = _blocks(self.AT, self.threads)

    def _product(self, blocks, rows, v):
        out = np.empty(rows)
        if self._pool is None:
            for a, b, M in blocks:
                out[a:b] = M @ v
            return out

        def work(blk):
            a, b, M = blk
            out[a:b] = M @ v

        list(self._pool.map(work, blocks))
        return out

    def Ax(self, x):
        return self._product(self._A_blocks, self.m, x)

    def ATy(self, y):
        return self._product(self._AT_blocks, self.n, y)

    def close(self):
        if self._pool is not None:
            self._pool.shutdown()
            self._pool = None
