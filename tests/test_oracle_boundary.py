"""The oracle and the CUDA path stay apart: the library never imports or includes the
oracle, the oracle never imports the library, and bench.py touches the oracle only in
its CPU-baseline and reference legs (__graft_entry__ builds it and smoke() checks with it)."""
import ast
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def imported_names(tree):
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name.split(".")[0], node
        elif isinstance(node, ast.ImportFrom) and node.module:
            yield node.module.split(".")[0], node


def test_library_never_uses_the_oracle():
    pkg = os.path.join(ROOT, "paper_1810_04201_gb300")
    for p in glob.glob(os.path.join(pkg, "*.py")):
        names = {n for n, _ in imported_names(ast.parse(open(p).read()))}
        assert "oracle" not in names, p
    for p in glob.glob(os.path.join(pkg, "csrc", "*")):
        assert not re.search(r'#include\s*[<"][^>"]*oracle', open(p).read()), p


def test_oracle_never_uses_the_library():
    for p in glob.glob(os.path.join(ROOT, "oracle", "*.py")):
        names = {n for n, _ in imported_names(ast.parse(open(p).read()))}
        assert "paper_1810_04201_gb300" not in names, p
    src = open(os.path.join(ROOT, "oracle", "wilson_oracle.c")).read()
    assert "wd.h" not in src and "csrc" not in src


def test_bench_touches_the_oracle_only_in_its_cpu_legs():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    owners = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for name, _ in imported_names(fn):
                if name == "oracle":
                    owners.add(fn.name)
    top = [n for n, node in imported_names(ast.Module(body=[s for s in tree.body
                                                             if isinstance(s, (ast.Import, ast.ImportFrom))],
                                                       type_ignores=[]))]
    assert "oracle" not in top
    assert owners <= {"cpu_baseline", "run_reference"}, owners
