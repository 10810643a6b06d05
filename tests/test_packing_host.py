"""Host logic of the lane packing, checked on the CPU (no GPU).

``packing_check.cpp`` is compiled against the library's packing code; it packs a matrix,
replays on the host what the warp lanes and the long-row pass compute from the stored
arrays, and compares with a plain CSR product (plus the layout's invariants: a row
permutation, consecutive slot rows within the per-slot budget, every nonzero stored once,
one end flag per row or piece).
"""
import os
import subprocess

import numpy as np
import pytest

import lpgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2601_07628_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    d = tmp_path_factory.mktemp("pack")
    exe = str(d / "packing_check")
    cuda_inc = "/usr/local/cuda/include"
    cmd = ["g++", "-O2", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I",
           cuda_inc, os.path.join(os.path.dirname(__file__), "packing_check.cpp"),
           os.path.join(CSRC, "packing.cpp"), os.path.join(CSRC, "preprocess.cpp"), "-o", exe,
           "-pthread"]
    subprocess.run(cmd, check=True)
    return exe, d


def run(checker, row_ptr, col, val, ncols, seed=0, offsets=None, threads=None, col_offsets=None,
        scaling_to=None):
    exe, d = checker
    rows = len(row_ptr) - 1
    x = np.random.default_rng(seed).standard_normal(ncols)
    path = str(d / f"m{seed}_{rows}_{ncols}.bin")
    with open(path, "wb") as f:
        np.array([rows, ncols, row_ptr[-1]], dtype=np.int64).tofile(f)
        np.asarray(row_ptr, dtype=np.int64).tofile(f)
        np.asarray(col, dtype=np.int32).tofile(f)
        np.asarray(val, dtype=np.float64).tofile(f)
        x.tofile(f)
    cmd = [exe, path] + ([",".join(str(int(o)) for o in offsets)] if offsets is not None else [])
    cmd += [",".join(str(int(o)) for o in col_offsets)] if col_offsets is not None else []
    env = dict(os.environ)
    if threads is not None:
        env["DPDLP_HOST_THREADS"] = str(threads)
    if scaling_to is not None:
        env["PACKING_CHECK_SCALING"] = str(scaling_to)
    out = subprocess.run(cmd, capture_output=True, text=True, env=env).stdout.strip()
    assert out.startswith("ok"), out
    return dict(kv.split("=") for kv in out.split()[1:])


LENGTHS = ([0, 1, 7, 8, 9, 31, 32, 33, 0, 0, 63, 64, 65, 255, 256, 257, 1000, 1023, 1024, 1025,
            4097, 9000, 0] + [5] * 600 + [0, 3000] + [17] * 200 + [1] * 900 + [0, 0])


def test_stress_rows(checker):
    lp = lpgen.row_length_stress_lp(11, LENGTHS, n=12000)
    st = run(checker, lp.row_ptr, lp.col, lp.val, lp.n)
    assert int(st["nlong"]) == sum(1 for L in LENGTHS if L > 32)


def test_transpose_of_stress(checker):
    """The CSC orientation of the same matrix (long columns of the transposed view)."""
    import scipy.sparse as sp

    lp = lpgen.row_length_stress_lp(12, LENGTHS, n=3000)
    A = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n)).T.tocsr()
    A.sort_indices()
    run(checker, A.indptr, A.indices, A.data, A.shape[1], seed=1)


def test_only_tiny_rows_and_empty(checker):
    """Many one-nonzero and empty rows: the per-slot row budget, not the lanes, limits."""
    rng = np.random.default_rng(3)
    lengths = rng.integers(0, 2, size=5000)
    lp = lpgen.row_length_stress_lp(13, lengths, n=50)
    run(checker, lp.row_ptr, lp.col, lp.val, lp.n, seed=2)


def test_empty_matrix_and_all_empty_rows(checker):
    run(checker, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0), 4, seed=3)
    run(checker, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), 4, seed=4)


def test_powerlaw_fill(checker):
    lp = lpgen.scaled_powerlaw_lp(1, 0.01)
    st = run(checker, lp.row_ptr, lp.col, lp.val, lp.n, seed=5)
    assert float(st["fill"]) > 0.85, st


def test_batch_packing(checker):
    """Several instances (block-diagonal stack, one of them empty): each instance's rows are
    packed into its own slots and keep their instance's index range."""
    import scipy.sparse as sp

    parts = [lpgen.row_length_stress_lp(20, LENGTHS, n=4000),
             lpgen.small_random_lp(21, n=300, m=0),
             lpgen.uneven_lp(22, 700),
             lpgen.row_length_stress_lp(23, [40, 0, 3, 33, 100, 1] * 20, n=500)]
    mats = [sp.csr_matrix((p.val, p.col, p.row_ptr), shape=(p.m, p.n)) for p in parts]
    B = sp.block_diag(mats).tocsr()
    B.sort_indices()
    offs = np.concatenate([[0], np.cumsum([p.m for p in parts])])
    st = run(checker, B.indptr, B.indices, B.data, B.shape[1], seed=7, offsets=offs)
    assert int(st["nlong"]) > 0
    # as the solver packs a batch: padding and empty rows gather their own instance's
    # first column (the checker verifies every stored index lies in its instance's
    # columns), and the products are unchanged
    coffs = np.concatenate([[0], np.cumsum([p.n for p in parts])])
    st2 = run(checker, B.indptr, B.indices, B.data, B.shape[1], seed=7, offsets=offs,
              col_offsets=coffs)
    assert st2["nlong"] == st["nlong"]


def test_cross_stress_fits_the_fused_body(checker):
    """The LP the fused-body GPU tests use: long rows of both classes the fused body runs
    (warp-class, more than 32 pieces, and thread-class) in A and in A^T, within 64 slots per
    orientation and without block-class rows (more than 256 pieces)."""
    import scipy.sparse as sp

    lp = lpgen.cross_stress_lp(5, [1500, 1100, 200, 40, 0, 1, 33] + [12] * 1493, 2000,
                               {5: 1200, 7: 600, 9: 40})
    A = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
    assert np.all(np.diff(lp.row_ptr)[:7] >= [1500, 1100, 200, 40, 0, 1, 33])
    assert np.all(np.diff(A.tocsc().indptr)[[5, 7, 9]] >= [1200, 600, 40])
    T = A.T.tocsr()
    T.sort_indices()
    for k, M in enumerate((A, T)):
        st = run(checker, M.indptr, M.indices, M.data, M.shape[1], seed=30 + k)
        lens = np.diff(M.indptr)
        assert int(st["slots"]) <= 64
        assert int(st["nlong"]) == int((lens > 32).sum())
        assert (lens > 32 * 32).any() and ((lens > 32) & (lens <= 32 * 32)).any()
        assert not (lens > 256 * 32).any()
    # planted optimum: feasible, and A^T y* + z* = c
    ax = A @ lp.x_star
    eq = lp.ctype == lpgen.EQ
    assert np.allclose(ax[eq], lp.b[eq]) and np.all(ax[~eq] <= lp.b[~eq] + 1e-12)
    assert np.allclose(A.T @ lp.y_star + lp.z_star, lp.c)


@pytest.mark.parametrize("case", ["stress", "batch", "powerlaw"])
def test_results_do_not_depend_on_host_threads(checker, case):
    """The load-time loops (transpose, permutation, packed arrays) run on host threads; every
    output is the same, bit for bit, with 1, 3 and 7 threads."""
    import scipy.sparse as sp

    offs = coffs = None
    if case == "stress":
        lp = lpgen.row_length_stress_lp(11, LENGTHS, n=12000)
        A = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
    elif case == "batch":
        parts = [lpgen.uneven_lp(40 + i, 300 + 97 * i) for i in range(12)]
        A = sp.block_diag([sp.csr_matrix((p.val, p.col, p.row_ptr), shape=(p.m, p.n))
                           for p in parts]).tocsr()
        A.sort_indices()
        offs = np.concatenate([[0], np.cumsum([p.m for p in parts])])
        coffs = np.concatenate([[0], np.cumsum([p.n for p in parts])])  # per-instance gathers
    else:
        lp = lpgen.scaled_powerlaw_lp(1, 0.01)
        A = sp.csr_matrix((lp.val, lp.col, lp.row_ptr), shape=(lp.m, lp.n))
    hashes = set()
    for t in (1, 3, 7):
        for M, off in ((A, offs), (A.T.tocsr(), None)):
            st = run(checker, M.indptr, M.indices, M.data, M.shape[1], seed=40 + t, offsets=off,
                     threads=t, col_offsets=coffs if off is not None else None)
            hashes.add((M.shape, st["hash"]))
    assert len(hashes) == 2, hashes


_M64 = (1 << 64) - 1


def _splitmix64(state):
    """SplitMix64 (Steele, Lea and Flood, 2014): advance the state by the golden-ratio
    increment, then two xor-shift-multiply rounds and a final xor-shift."""
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def _block_permutation(length, block, seed):
    """Reading O17: Fisher-Yates over the whole blocks (i from the last block down to 1, j =
    the next SplitMix64 output mod (i + 1)), rows keeping their order inside a block, the
    trailing partial block in place; new position k holds old row perm[k]."""
    perm = list(range(length))
    if length <= block:
        return perm
    nfull = length // block
    order = list(range(nfull))
    state = seed
    for i in range(nfull - 1, 0, -1):
        state, r = _splitmix64(state)
        j = r % (i + 1)
        order[i], order[j] = order[j], order[i]
    for b in range(nfull):
        for t in range(block):
            perm[b * block + t] = order[b] * block + t
    return perm


def test_block_permutation_is_splitmix64_fisher_yates(checker):
    """The solver's block permutation (host C++) against the reading written out in Python
    from the published SplitMix64 definition, whose first output from state 0 is
    0xE220A8397B1DCDAF; row and column seeds of a single LP and of batch instances."""
    assert _splitmix64(0)[1] == 0xE220A8397B1DCDAF
    exe, _ = checker
    for length, block, seed in ((1000, 256, 1), (1000, 256, 2), (100_003, 256, 1), (100_003, 256, 8),
                                (512, 256, 5), (255, 256, 1), (7, 3, 7)):
        out = subprocess.run([exe, "--perm", str(length), str(block), str(seed)], capture_output=True,
                             text=True, check=True).stdout.strip()
        got = [int(v) for v in out.split(",")] if out else []
        assert got == _block_permutation(length, block, seed), (length, block, seed)


def test_host_preconditioner_matches_the_oracle(checker, tmp_path):
    """The solver's host preconditioner (C++) computes the oracle's factors exactly: 10 Ruiz
    passes, then one Pock-Chambolle pass, each factor the power of two nearest to
    1/sqrt(row or column norm) (reading O15), on a matrix whose entries span twelve
    decades."""
    from oracle import pdhg as O
    from oracle import precond as P
    import test_precond_oracle as pp

    A = pp.badly_scaled(5)
    m, n = A.shape
    path = tmp_path / "scaling.bin"
    run(checker, A.indptr, A.indices, A.data, n, seed=50, scaling_to=path)
    d = np.fromfile(path, dtype=np.float64)
    lp = O.OracleLP(n, m, np.ones(n), A.indptr, A.indices, A.data, -np.ones(m), np.ones(m),
                    np.zeros(n), np.full(n, 3.0))
    dr, dc = P.scale_factors(lp)
    assert d.shape == (m + n,)
    assert np.array_equal(d[:m], dr) and np.array_equal(d[m:], dc)
    assert dr.min() < 1e-2 and dr.max() > 1e2  # the factors do vary
