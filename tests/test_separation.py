"""The CUDA path and the oracle share no code and neither imports the other.

The product package (Python binding, kernels, headers, input generators) must
not import, include or load anything under oracle/, and the oracle must not
use the package or the library's headers.  bench.py may run the oracle only
for its CPU baseline and its reference arm, from functions of its own, never
at import.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2007_14401_gb300")
ORACLE = os.path.join(ROOT, "oracle")
SRC_EXT = (".py", ".cu", ".cuh", ".h", ".c", ".cpp")


def sources(top):
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if not x.startswith(("_", "."))]
        for f in files:
            if f.endswith(SRC_EXT):
                yield os.path.join(d, f)


def code_of(path):
    """The file without comments and docstrings (so prose may name the oracle)."""
    text = open(path, encoding="utf-8").read()
    if path.endswith(".py"):
        tree = ast.parse(text)
        return "\n".join(ast.unparse(n) for n in tree.body
                         if not (isinstance(n, ast.Expr) and isinstance(n.value, ast.Constant)))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.sub(r"//[^\n]*", "", text)


def test_package_does_not_use_the_oracle():
    bad = re.compile(r"\bimport\s+oracle\b|\bfrom\s+oracle\b|gcb_oracle|[\"']oracle[/\"']")
    hits = [p for p in sources(PKG) if bad.search(code_of(p))]
    assert not hits, hits


def test_oracle_does_not_use_the_package():
    bad = re.compile(r"paper_2007_14401_gb300|gcb_internal\.h|gcb_device\.cuh|push_sr\.cuh|"
                     r"sort_sr\.h|libgcb|#include\s+\"gcb\.h\"")
    hits = [p for p in sources(ORACLE) if bad.search(code_of(p))]
    assert not hits, hits


def test_bench_runs_the_oracle_only_from_its_baseline_helpers():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py"), encoding="utf-8").read())
    for node in tree.body:                      # nothing at import time
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            names = [a.name for a in node.names] + [getattr(node, "module", None) or ""]
            assert not any(n.split(".")[0] == "oracle" for n in names)
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for n in ast.walk(fn):
                if isinstance(n, (ast.Import, ast.ImportFrom)):
                    mods = [a.name for a in n.names] + [getattr(n, "module", None) or ""]
                    if any(m.split(".")[0] == "oracle" for m in mods):
                        users.add(fn.name)
    assert users and users <= {"_oracle_ks", "_oracle_for"}, users
