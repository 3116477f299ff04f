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


def test_launch_shape_is_host_only_and_consistent():
    from paper_2510_15649_gb300 import ladlasso as ll

    class Pr:  # the two fields launch_shape reads
        def __init__(self, P, n_max):
            self.P, self.n_max = P, n_max

    g, f, m = ll.launch_shape(Pr(32, 2000))
    assert g == 32 and 1 <= f <= 16 and m >= 8192
    # fewer rows per fit -> at least as many fits per block
    g2, f2, _ = ll.launch_shape(Pr(32, 500))
    assert g2 == 32 and f2 >= f
    # the hint caps the count and never raises it
    assert ll.launch_shape(Pr(32, 2000), ll.Launch(32, 3))[1] == min(3, f)
    assert ll.launch_shape(Pr(32, 2000), ll.Launch(32, 99))[1] == f
    # beyond 8192 rows: one block per fit, up to the shared-memory row limit
    g3, f3, m3 = ll.launch_shape(Pr(128, 20000))
    assert g3 == 512 and f3 == 1 and m3 >= 20000
    assert ll.launch_shape(Pr(32, 2000), ll.Launch(512, 0))[0] == 512
    # n_max beyond the one-warp limit with an explicit one-warp request
    g4, f4, m4 = ll.launch_shape(Pr(32, 50000), ll.Launch(32, 0))
    assert g4 == 32 and m4 < 50000
    # wide problems: the automatic shape takes one block per fit when a
    # warp's share of shared memory cannot hold n_max rows but a block's can
    g5, _, m5 = ll.launch_shape(Pr(180, 7000))
    assert g5 == 512 and m5 >= 7000
    assert ll.launch_shape(Pr(180, 7000), ll.Launch(32, 0))[2] < 7000
    assert ll.launch_shape(Pr(180, 5000))[0] == 32  # a warp still holds it
    # two or four warps per fit: fewer fits per block (at most 512 threads),
    # a little less room for rows than one warp (larger selection buffers)
    for gt in (64, 128):
        g6, f6, m6 = ll.launch_shape(Pr(32, 2000), ll.Launch(gt, 0))
        assert g6 == gt and 1 <= f6 <= 512 // gt and f6 <= f and 8192 <= m6 <= m
    # invalid shapes
    import pytest
    for bad in (96, 256, 1024):
        with pytest.raises(ll.LadLassoError):
            ll.launch_shape(Pr(32, 2000), ll.Launch(bad, 0))


def test_documented_option_defaults_match_the_library():
    # each ladlasso_opts field's comment in include/ladlasso.h ends with its
    # default in parentheses; ladlasso_default_opts must fill exactly those
    from paper_2510_15649_gb300 import ladlasso
    src = open(os.path.join(ROOT, "include", "ladlasso.h")).read()
    body = src[src.index("typedef struct ladlasso_opts"):src.index("} ladlasso_opts;")]
    fields = re.findall(r"(?:float|int32_t)\s+(\w+);(.*?)(?=(?:float|int32_t)\s+\w+;|\Z)", body, re.S)
    o = ladlasso.default_opts()
    assert len(fields) == len(o._fields_)
    for name, comment in fields:
        doc = re.findall(r"\(([-0-9.e]+)\)", comment)
        assert doc, name
        assert abs(float(doc[-1]) - getattr(o, name)) <= 1e-6 * max(1.0, abs(float(doc[-1]))), name
