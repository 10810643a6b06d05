"""The allocation-free SpMV entry point against the oracle's A x (needs a GB300).

``dpdlp_csr_spmv_noalloc`` serves callers that cannot allocate device memory where they
need a product -- a framework whose own pool has reserved the device's memory, or a
latency-critical loop that must not stall on the allocator -- by keeping its only scratch
in one fixed device array.  This test calls it through the C ABI twice in a row (an LP
with long rows that span many thread-block parts, then a smaller LP) and compares each
result with the oracle's A x and with the solver's own ``dpdlp_apply_A``, at the tolerance
of the other SpMV tests; it then checks that 100 further calls leave the device's free
memory unchanged.  The file is named to run after every other test.
"""
import numpy as np
import pytest

import lpgen
from oracle import pdhg as O

pytestmark = pytest.mark.gpu


def _lps():
    lengths = [0, 3, 9000, 0, 0, 70000, 5, 257, 4097] + [11] * 500 + [0, 2048, 30000, 0]
    return [lpgen.row_length_stress_lp(21, lengths, n=80000), lpgen.small_random_lp(0)]


def _device_csr(lp, torch, dev):
    rp = torch.from_numpy(lp.row_ptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(lp.col.astype(np.int32)).to(dev)
    va = torch.from_numpy(np.ascontiguousarray(lp.val)).to(dev)
    return rp, ci, va


def _close(got, want, x):
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(x).max() * 100)


def test_noalloc_spmv_matches_oracle_and_apply_A():
    import torch

    from paper_2601_07628_gb300 import build
    from paper_2601_07628_gb300.dpdlp import Solver, csr_spmv_noalloc

    build()
    torch.cuda.init()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(4)
    for lp in _lps():  # two calls in a row, different sizes
        x = rng.standard_normal(lp.n)
        want = O.OracleLP.from_lpgen(lp).Ax(x)
        with Solver(0) as s:
            s.load(lp)
            solver_ax = s.apply_A(x)
        rp, ci, va = _device_csr(lp, torch, dev)
        xd = torch.from_numpy(x).to(dev)
        y = torch.full((lp.m,), np.nan, dtype=torch.float64, device=dev)
        assert csr_spmv_noalloc(rp, ci, va, xd, y, lp.n) == 0
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        _close(got, want, x)
        _close(got, solver_ax, x)


def test_noalloc_spmv_allocates_nothing():
    """Free device memory (cudaMemGetInfo) is the same before and after 100 calls, with
    every tensor allocated beforehand and the caching allocator left alone in between."""
    import torch

    from paper_2601_07628_gb300 import build
    from paper_2601_07628_gb300.dpdlp import csr_spmv_noalloc

    build()
    torch.cuda.init()
    dev = torch.device("cuda", 0)
    lp = _lps()[0]
    x = np.random.default_rng(5).standard_normal(lp.n)
    rp, ci, va = _device_csr(lp, torch, dev)
    xd = torch.from_numpy(x).to(dev)
    y = torch.empty(lp.m, dtype=torch.float64, device=dev)
    assert csr_spmv_noalloc(rp, ci, va, xd, y, lp.n) == 0  # kernels loaded, address looked up
    torch.cuda.synchronize()
    first = y.cpu().numpy()
    free0, _ = torch.cuda.mem_get_info(0)
    for _ in range(100):
        assert csr_spmv_noalloc(rp, ci, va, xd, y, lp.n) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0, (free0, free1)
    assert np.array_equal(y.cpu().numpy(), first)  # reruns are bitwise identical


def test_noalloc_spmv_rejects_bad_arguments():
    import ctypes as C

    import torch

    from paper_2601_07628_gb300 import build
    from paper_2601_07628_gb300.dpdlp import csr_spmv_noalloc, load_library

    build()
    lib = load_library()
    dummy = C.c_void_p(16)  # never dereferenced: the size check comes first
    assert lib.dpdlp_csr_spmv_noalloc(10, 10, (1 << 30) + 1, dummy, dummy, dummy, dummy, dummy,
                                      None) == -6
    assert lib.dpdlp_csr_spmv_noalloc(-1, 10, 0, dummy, dummy, dummy, dummy, dummy, None) == -1
    dev = torch.device("cuda", 0)
    lp = lpgen.small_random_lp(0, n=20, m=10, nnz_per_col=2)
    rp, ci, va = _device_csr(lp, torch, dev)
    xd = torch.zeros(lp.n, dtype=torch.float64, device=dev)
    y = torch.zeros(lp.m, dtype=torch.float64, device=dev)
    # wrong index type, wrong value type, a host tensor, a short output: refused before the call
    assert csr_spmv_noalloc(rp.long(), ci, va, xd, y, lp.n) == -1
    assert csr_spmv_noalloc(rp, ci, va.float(), xd, y, lp.n) == -1
    assert csr_spmv_noalloc(rp, ci, va, xd.cpu(), y, lp.n) == -1
    assert csr_spmv_noalloc(rp, ci, va, xd, y[:-1], lp.n) == -1
