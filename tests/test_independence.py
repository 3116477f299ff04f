"""The oracle and the CUDA path share no code: the product (the package,
its CUDA sources and the C header) never imports, includes or links the
oracle; the oracle never includes the library's headers or imports the
package; bench.py reaches the oracle only inside its CPU legs (the
reference arm, the sampled parity check and the CPU baseline), never at
module level.  Checked on the source text and the syntax tree."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2510_15649_gb300")


def _imports(tree):
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [a.name.split(".")[0] for a in node.names]
        elif isinstance(node, ast.ImportFrom) and node.module:
            out.append(node.module.split(".")[0])
    return out


def test_product_python_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "*.py")):
        assert "oracle" not in _imports(ast.parse(open(path).read())), path


def test_product_native_code_never_includes_or_calls_the_oracle():
    files = glob.glob(os.path.join(PKG, "csrc", "*")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert files
    for path in files:
        src = open(path).read()
        assert not re.search(r'#include\s*[<"][^>"]*oracle', src), path
        assert not re.search(r"\borc_\w+\s*\(", src), path
    build = open(os.path.join(PKG, "build.py")).read()
    assert "oracle" not in build and "liboracle" not in build


def test_oracle_never_uses_the_product():
    src = open(os.path.join(ROOT, "oracle", "ladlasso_oracle.c")).read()
    assert not re.search(r'#include\s*"', src)  # system headers only
    assert "ladlasso_" not in re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    tree = ast.parse(open(os.path.join(ROOT, "oracle", "__init__.py")).read())
    assert set(_imports(tree)) <= {"__future__", "ctypes", "os", "subprocess", "numpy"}


def test_bench_imports_the_oracle_only_inside_its_cpu_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert "oracle" not in _imports(ast.Module(body=top, type_ignores=[]))
    src = open(os.path.join(ROOT, "bench.py")).read()
    # each import of the oracle sits in a block that names one of the CPU legs
    for m in re.finditer(r"^( *)import oracle$", src, re.M):
        before = src[:m.start()].split("\n")[-25:]
        ctx = "\n".join(before)
        assert re.search(r"run_reference|parity|cpu_baseline|CPU oracle", ctx), ctx[-400:]
