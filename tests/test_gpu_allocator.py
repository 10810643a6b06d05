"""Device allocator hook: the LP's buffers come from torch's caching allocator."""
import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session")
def Solver():
    from paper_2601_07628_gb300 import build, dpdlp

    build()
    return dpdlp.Solver


def test_torch_allocator_backs_device_memory(Solver):
    import torch

    lp = lpgen.small_random_lp(0)
    a = Solver()
    a.load(lp)
    a.solve(1e-6, 100_000)
    xa, ya = a.solution()
    a.close()
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    b = Solver()
    b.use_torch_allocator()
    b.load(lp)
    assert torch.cuda.memory_allocated() - base >= b.info()["device_bytes"]
    b.solve(1e-6, 100_000)
    xb, yb = b.solution()
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)
    b.load(lpgen.small_random_lp(1))  # the previous LP's buffers go back first
    b.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_allocator_arguments(Solver):
    from paper_2601_07628_gb300 import dpdlp

    s = Solver()
    with pytest.raises(dpdlp.DpdlpError):  # one function without the other
        s._check(s.lib.dpdlp_set_allocator(s.h, dpdlp.ALLOC_FN(lambda n, c: None), dpdlp.RELEASE_FN(), None))
    s.use_torch_allocator()
    s.load(lpgen.small_random_lp(2, n=200, m=100))
    s.use_torch_allocator(False)  # unloads; back to cudaMalloc
    with pytest.raises(dpdlp.DpdlpError):
        s.solve(1e-4, 100)  # nothing loaded
    s.load(lpgen.small_random_lp(2, n=200, m=100))
    assert s.solve(1e-4, 100_000) == 0
    s.close()
