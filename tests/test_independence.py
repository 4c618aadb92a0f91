"""The oracle and the CUDA path share no code.

The oracle is the independent check of every GPU result, so neither side may
import, include or call the other; only seeded_inputs.py (random draws, none
of the method's arithmetic) serves both.  These checks read the sources as
text and need no GPU.
"""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2410_09497_gb300")


def _files(top, exts):
    for d, _, fs in os.walk(top):
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out


def test_product_does_not_use_the_oracle():
    for p in _files(PKG, (".py",)):
        assert "oracle" not in _imports(p), p
    for p in list(_files(PKG, (".cu", ".cuh", ".cpp", ".h"))) + list(_files(os.path.join(ROOT, "include"), (".h",))):
        text = open(p).read()
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", text), p


def test_oracle_does_not_use_the_product():
    for p in _files(os.path.join(ROOT, "oracle"), (".py",)):
        imp = _imports(p)
        assert "paper_2410_09497_gb300" not in imp and "ctypes" not in imp, p
        assert "libstokesmg" not in open(p).read(), p


def test_seeded_inputs_hold_no_method_code():
    imp = _imports(os.path.join(ROOT, "seeded_inputs.py"))
    assert not imp & {"oracle", "paper_2410_09497_gb300", "scipy"}, imp
