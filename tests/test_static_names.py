"""Every global name a Python file of the repository reads is defined in
that file or is a builtin.  Much of this code (the GPU tests, the bench's
GPU arms, the binding's launch paths) only runs on a GPU, so a misspelt or
deleted helper would otherwise surface there first; the symbol tables catch
it on the CPU."""
import builtins
import glob
import os
import symtable

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = sorted(
    [os.path.relpath(p, ROOT) for p in glob.glob(os.path.join(ROOT, "paper_2510_15649_gb300", "*.py"))]
    + [os.path.relpath(p, ROOT) for p in glob.glob(os.path.join(ROOT, "tests", "*.py"))]
    + ["oracle/__init__.py", "bench.py", "__graft_entry__.py"])
IMPLICIT = {"__file__", "__name__", "__doc__", "__builtins__", "__spec__"}


def _read_globals(table, out):
    for s in table.get_symbols():
        if s.is_global() and s.is_referenced():
            out.add(s.get_name())
    for child in table.get_children():
        _read_globals(child, out)


@pytest.mark.parametrize("path", FILES)
def test_every_global_read_is_defined(path):
    src = open(os.path.join(ROOT, path)).read()
    top = symtable.symtable(src, path, "exec")
    read = set()
    _read_globals(top, read)
    defined = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    missing = sorted(n for n in read - defined - IMPLICIT if not hasattr(builtins, n))
    assert not missing, f"{path}: {missing}"
