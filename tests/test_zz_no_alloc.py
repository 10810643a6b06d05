"""The allocation-free SpMV entry point agrees with the solver's own A x.

``dpdlp_csr_spmv_noalloc`` serves callers that cannot allocate device memory where they
need a product (for example while recording a CUDA graph, or inside a framework whose pool
owns all device memory): it keeps its scratch in one fixed device array.  This test calls
it through the C ABI twice in a row -- on an LP with long rows that span many thread-block
parts, then on a smaller LP -- and compares each result with ``dpdlp_apply_A`` (same
tolerance as the other SpMV tests).  The file is named to run after every other test.
"""
import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu


def _lps():
    lengths = [0, 3, 9000, 0, 0, 70000, 5, 257, 4097] + [11] * 500 + [0, 2048, 30000, 0]
    return [lpgen.row_length_stress_lp(21, lengths, n=80000), lpgen.small_random_lp(0)]


def test_noalloc_spmv_matches_apply_A():
    import torch

    from paper_2601_07628_gb300 import build
    from paper_2601_07628_gb300.dpdlp import Solver, csr_spmv_noalloc

    build()
    torch.cuda.init()
    rng = np.random.default_rng(4)
    for lp in _lps():  # two calls in a row, different sizes
        x = rng.standard_normal(lp.n)
        with Solver(0) as s:
            s.load(lp)
            want = s.apply_A(x)
        dev = torch.device("cuda", 0)
        rp = torch.from_numpy(lp.row_ptr.astype(np.int32)).to(dev)
        ci = torch.from_numpy(lp.col.astype(np.int32)).to(dev)
        va = torch.from_numpy(lp.val).to(dev)
        xd = torch.from_numpy(x).to(dev)
        y = torch.full((lp.m,), np.nan, dtype=torch.float64, device=dev)
        assert csr_spmv_noalloc(rp, ci, va, xd, y, lp.n) == 0
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * np.abs(x).max() * 100)


def test_noalloc_spmv_rejects_sizes_beyond_its_scratch():
    import ctypes as C

    from paper_2601_07628_gb300 import build
    from paper_2601_07628_gb300.dpdlp import load_library

    build()
    lib = load_library()
    dummy = C.c_void_p(16)  # never dereferenced: the size check comes first
    assert lib.dpdlp_csr_spmv_noalloc(10, 10, (1 << 30) + 1, dummy, dummy, dummy, dummy, dummy,
                                      None) == -6
    assert lib.dpdlp_csr_spmv_noalloc(-1, 10, 0, dummy, dummy, dummy, dummy, dummy, None) == -1
