"""The C ABI library loads and exports every entry point its header declares (no GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in ("dpdlp.h", "dpdlp_gnn.h")]


def declared_symbols():
    out = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        out |= set(re.findall(r"\b(dpdlp_[a-z_A-Z0-9]+)\s*\(", text))
    return sorted(out)


@pytest.fixture(scope="module")
def lib():
    from paper_2601_07628_gb300 import build, dpdlp

    build()
    return dpdlp.load_library()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("dpdlp_load_lp", "dpdlp_solve", "dpdlp_get_solution", "dpdlp_get_kkt"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2601_07628_gb300 import dpdlp

    out = subprocess.run(["nm", "-D", "--defined-only", dpdlp.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    from paper_2601_07628_gb300 import gnn

    for s in declared_symbols():
        assert hasattr(lib, s)
        assert s in dpdlp.EXPORTS or s in gnn.EXPORTS, f"binding lacks a signature for {s}"


def test_gnn_param_count_matches_reference_layout(lib):
    from oracle import gnn as G
    from paper_2601_07628_gb300 import gnn

    assert gnn.param_count() == G.param_count()
    assert gnn.init_params(0).shape == (G.param_count(),)


def test_struct_layouts_match_header(lib):
    """ctypes mirrors of the ABI structs have the sizes a C compiler gives them."""
    import ctypes as C
    import tempfile

    from paper_2601_07628_gb300 import dpdlp

    src = r"""
#include <stdio.h>
#include "dpdlp.h"
int main(void){printf("%zu %zu %zu %zu\n", sizeof(dpdlp_kkt_t), sizeof(dpdlp_trace_t),
 sizeof(dpdlp_scalar_state_t), sizeof(dpdlp_info_t));return 0;}
"""
    with tempfile.TemporaryDirectory() as d:
        cf = os.path.join(d, "s.c")
        open(cf, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), cf, "-o", exe], check=True)
        sizes = list(map(int, subprocess.run([exe], capture_output=True, text=True).stdout.split()))
    assert sizes == [C.sizeof(dpdlp.KKT), C.sizeof(dpdlp.Trace), C.sizeof(dpdlp.ScalarState),
                     C.sizeof(dpdlp.Info)]


def test_error_paths_without_device(lib):
    """Calls on a NULL handle fail with DPDLP_ERR_INVALID and never crash."""
    import ctypes as C

    assert lib.dpdlp_set_param(None, b"eta", 1.0) == -1
    assert lib.dpdlp_solve(None, 1e-8, 10) == -1
    assert lib.dpdlp_get_solution(None, None, None) == -1
    lib.dpdlp_destroy(None)
    assert lib.dpdlp_last_error(None) == b"null handle"
