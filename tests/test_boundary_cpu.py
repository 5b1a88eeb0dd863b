"""The product path and the oracle stay apart, and the product fails loudly
without its compiled library.

- No source of the package (the ctypes binding, its build script, the CUDA and
  C++ translation units) names the oracle module.
- The benchmark imports the oracle only inside its CPU-baseline leg
  (`cpu_leg`), never at module level or on the GPU path.
- The binding raises ImportError when libflz.so is absent instead of falling
  back to any CPU computation.
"""

import ast
import glob
import importlib
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2409_15053_gb300")


def test_package_sources_never_name_the_oracle():
    files = glob.glob(os.path.join(PKG, "*.py")) + glob.glob(os.path.join(PKG, "csrc", "*"))
    files += glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert len(files) > 10
    for f in files:
        with open(f, encoding="utf-8") as fh:
            text = fh.read()
        assert not re.search(r"\boracle\b", text), f"{os.path.relpath(f, ROOT)} names the oracle"


def _oracle_imports(tree):
    """(enclosing function name or None, line) of every import of the oracle package."""
    found = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) else fn
            if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                found.append((fn, child.lineno))
            if isinstance(child, ast.ImportFrom) and (child.module or "").split(".")[0] == "oracle":
                found.append((fn, child.lineno))
            visit(child, name)

    visit(tree, None)
    return found


def test_benchmark_imports_the_oracle_only_in_its_cpu_leg():
    with open(os.path.join(ROOT, "bench.py"), encoding="utf-8") as fh:
        tree = ast.parse(fh.read())
    imports = _oracle_imports(tree)
    assert imports, "the CPU-baseline leg times the oracle"
    assert {fn for fn, _ in imports} == {"cpu_leg"}, imports


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    flz = importlib.import_module("paper_2409_15053_gb300")
    monkeypatch.setattr(flz, "_lib", None)
    monkeypatch.setattr(flz, "LIB_PATH", str(tmp_path / "libflz.so"))
    try:
        flz.lib()
    except ImportError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("lib() returned without a library")
