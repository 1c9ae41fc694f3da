"""The oracle and the CUDA path share no code: the package never imports the
oracle, the oracle never imports the package, and the seeded input generators
(workloads/) import neither.  The library's C/CUDA sources include only their own
headers.  Checked on the source text, so it runs without a GPU."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_2312_07725_gb300"


def _py_files(sub):
    for dirpath, _, files in os.walk(os.path.join(ROOT, sub)):
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(dirpath, f)


def _imported_roots(path):
    tree = ast.parse(open(path).read())
    roots = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            roots.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            roots.add(node.module.split(".")[0])
    return roots


def test_package_does_not_import_the_oracle():
    for f in _py_files(PKG):
        assert "oracle" not in _imported_roots(f), f


def test_oracle_does_not_import_the_package():
    for f in _py_files("oracle"):
        assert PKG not in _imported_roots(f), f


def test_workloads_import_neither_side():
    for f in _py_files("workloads"):
        roots = _imported_roots(f)
        assert "oracle" not in roots and PKG not in roots, f


def test_cuda_sources_include_only_their_own_headers():
    csrc = os.path.join(ROOT, PKG, "csrc")
    own = set(os.listdir(csrc)) | {"nsfr.h"}
    for f in os.listdir(csrc):
        if not f.endswith((".cu", ".cuh", ".cpp", ".h")):
            continue
        for inc in re.findall(r'#include\s+"([^"]+)"', open(os.path.join(csrc, f)).read()):
            assert os.path.basename(inc) in own, (f, inc)
            assert "oracle" not in inc, (f, inc)
