"""Every repository path that README.md name in backticks
exists (`csrc/...` is relative to the package), so the documents cannot
point at files that were renamed or removed."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2510_15649_gb300"


def _paths(doc):
    s = open(os.path.join(ROOT, doc)).read()
    found = set(re.findall(
        r"`((?:tests|paper_2510_15649_gb300|profiles|include|oracle|csrc)/[A-Za-z0-9_./-]+?)"
        r"(?:::[A-Za-z0-9_\[\]]+)?`", s))
    found |= {p for p in re.findall(r"`([A-Za-z0-9_./-]+\.(?:py|cu|cuh|h|c|md))`", s) if "/" in p}
    return sorted(found)


@pytest.mark.parametrize("doc", ["DESIGN.md", "README.md"])
def test_named_paths_exist(doc):
    paths = _paths(doc)
    assert paths, doc
    missing = [p for p in paths
               if not os.path.exists(os.path.join(ROOT, p)) and
               not os.path.exists(os.path.join(ROOT, PKG, p))]
    assert not missing, (doc, missing)


@pytest.mark.parametrize("doc", ["DESIGN.md", "README.md"])
def test_named_tests_exist(doc):
    s = open(os.path.join(ROOT, doc)).read()
    refs = re.findall(r"`((?:tests/)?test_[A-Za-z0-9_]+\.py)::([A-Za-z0-9_]+)", s)
    missing = []
    for path, name in refs:
        full = os.path.join(ROOT, path if path.startswith("tests/") else os.path.join("tests", path))
        if not os.path.exists(full) or f"def {name}(" not in open(full).read():
            missing.append(f"{path}::{name}")
    assert not missing, (doc, missing)


@pytest.mark.parametrize("doc", sorted(os.path.relpath(p, ROOT)
                                       for p in glob.glob(os.path.join(ROOT, "profiles", "*.md"))))
def test_profile_summaries_name_committed_files_only(doc):
    s = open(os.path.join(ROOT, doc)).read()
    assert "_work/" not in s and "gpurun" not in s, doc
    assert "--clock-control none" in s, doc  # every capture left the clocks alone
    assert "bench.py" in s, doc              # the command runs a committed script
    for p in _paths(doc):
        assert os.path.exists(os.path.join(ROOT, p)) or os.path.exists(os.path.join(ROOT, PKG, p)), p
