"""The oracle and the CUDA path share no code, and the product never runs
the oracle: a static check of the sources.

- Nothing in the package (Python binding, CUDA sources, build script) or in
  the public header imports, includes or loads anything of ``oracle/``.
- Nothing in ``oracle/`` imports, includes or loads the package or its header.
- The seeded input generators (``scenes/``), which both sides use, import
  neither.
- ``bench.py`` imports the oracle only inside its CPU-baseline and
  reference-arm functions; ``__graft_entry__.py`` only inside ``build``
  (which compiles it) and ``smoke`` (which checks against it)."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SOURCE_EXT = (".py", ".cu", ".cuh", ".h", ".c", ".cpp")


def sources(sub):
    top = os.path.join(ROOT, sub)
    for dirpath, dirnames, files in os.walk(top):
        dirnames[:] = [d for d in dirnames if not d.startswith(("_lib", "__pycache__", "_build"))]
        for f in files:
            if f.endswith(SOURCE_EXT):
                yield os.path.join(dirpath, f)


ORACLE_REF = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b|#\s*include\s*[<\"].*oracle)|libcvo_oracle|orc_[a-z]+\(",
                        re.M)
PACKAGE_REF = re.compile(r"paper_2012_03683_gb300|#\s*include\s*[<\"][^>\"]*cvo(_internal)?\.(h|cuh)|libcvo\.so", re.M)


@pytest.mark.parametrize("sub", ["paper_2012_03683_gb300", "include"])
def test_product_does_not_reference_the_oracle(sub):
    files = list(sources(sub))
    assert files
    for f in files:
        assert not ORACLE_REF.search(open(f).read()), f


def test_oracle_does_not_reference_the_product():
    files = list(sources("oracle"))
    assert any(f.endswith(".c") for f in files)
    for f in files:
        assert not PACKAGE_REF.search(open(f).read()), f


def test_input_generators_reference_neither():
    for f in sources("scenes"):
        text = open(f).read()
        assert not ORACLE_REF.search(text) and not PACKAGE_REF.search(text), f


def oracle_imports(path):
    """(enclosing top-level function or None, line) of every oracle import."""
    tree = ast.parse(open(path).read())
    found = []

    def visit(node, func):
        for child in ast.iter_child_nodes(node):
            f = child.name if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) and func is None else func
            if isinstance(child, ast.Import) and any(a.name.split(".")[0] == "oracle" for a in child.names):
                found.append((func, child.lineno))
            elif isinstance(child, ast.ImportFrom) and (child.module or "").split(".")[0] == "oracle":
                found.append((func, child.lineno))
            visit(child, f)

    visit(tree, None)
    return found


@pytest.mark.parametrize("name,allowed", [("bench.py", {"cpu_baseline", "run_reference"}),
                                          ("__graft_entry__.py", {"build", "smoke"})])
def test_oracle_imported_only_where_allowed(name, allowed):
    found = oracle_imports(os.path.join(ROOT, name))
    assert found, name
    for func, line in found:
        assert func in allowed, (name, func, line)
