"""The C-ABI library builds for sm_103a, loads, and exports every entry
point declared in include/ladlasso.h (no GPU needed: no compute calls)."""
import ctypes as C
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "ladlasso.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ladlasso_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2510_15649_gb300 import build, ladlasso
    build.build()
    lib = C.CDLL(ladlasso.LIB_PATH)
    names = declared()
    assert len(names) >= 8
    for nm in names:
        assert hasattr(lib, nm), nm
    assert sorted(ladlasso.SYMBOLS) == names


def test_host_only_entry_points():
    from paper_2510_15649_gb300 import ladlasso
    L = ladlasso.lib()
    o = ladlasso.default_opts()
    assert abs(o.tol_move - 1e-6) < 1e-12 and o.chop == 1 and o.polish == 1
    assert L.ladlasso_workspace_size(10, 8, 1000, 4) > 1000 * 8 * 4
    assert L.ladlasso_workspace_size(-1, 8, 1000, 4) == 0
    assert L.ladlasso_workspace_size(1, 0, 10, 1) == 0
    assert L.ladlasso_status_string(0) == b"ok"
    assert L.ladlasso_status_string(-4).startswith(b"workspace")
    # invalid host arguments are rejected before any CUDA call
    assert L.ladlasso_lambda_path(None, -1, 1, 0.5, None, None) == ladlasso.ERR_INVALID
    assert L.ladlasso_fit_batched(None, None, None, None, None, None, None, None, None) == ladlasso.ERR_INVALID
