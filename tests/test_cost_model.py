"""The cost model of Eq. cost_model reproduces the paper's worked examples (Appendix E.3)."""
import os

from paper_2601_07628_gb300.costmodel import kernel_bytes, t_step

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cost_model_examples.txt")


def _rows():
    rows, speed = [], {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "speedup":
            speed[f[1]] = (float(f[2]), float(f[3]))
        else:
            rows.append((f[0], *map(int, f[1:6]), *map(float, f[6:])))
    return rows, speed


def test_worked_examples():
    rows, speed = _rows()
    assert len(rows) == 6
    single = {}
    for name, m, n, nnz, R, C, spmv, vec, net, lat, total in rows:
        t = t_step(m, n, nnz, R, C)
        for got, want in ((t.spmv_s, spmv), (t.vec_s, vec), (t.net_s, net), (t.latency_s, lat)):
            assert abs(got * 1e3 - want) <= 0.0005 + 1e-12, (name, R, C, got * 1e3, want)
        # the printed totals add the rounded terms, so they may differ from the exact sum
        # in the last digit
        assert abs(t.total_s * 1e3 - total) <= 0.0015, (name, R, C, t.total_s * 1e3, total)
        if R * C == 1:
            single[name] = t.total_s
        else:
            s = single[name] / t.total_s
            want = speed[name][0 if R * C == 4 else 1]
            assert abs(s - want) <= 0.006, (name, R * C, s, want)


def test_kernel_bytes_powerlaw_workload():
    """4M x 2M with 40M nonzeros: about 1.34 GB of algorithmic traffic per iteration."""
    b = kernel_bytes(4_000_000, 2_000_000, 40_000_000)
    assert b["iteration"] == 24 * 40_000_000 + 4 * 4_000_001 + 4 * 2_000_001 + 8 * 2_000_000 \
        + 56 * 4_000_000 + 8 * 4_000_000 + 40 * 2_000_000
    assert 1.33e9 < b["iteration"] < 1.36e9
