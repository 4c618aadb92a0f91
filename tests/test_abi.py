"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(stk_[A-Za-z0-9_]+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2410_09497_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_symbols()
    for required in ["stk_setup", "stk_destroy", "stk_apply", "stk_residual", "stk_layout", "stk_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_arguments_fail_without_gpu(lib):
    P = ctypes.c_void_p()
    lib.stk_setup.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    lib.stk_last_error.restype = ctypes.c_char_p
    assert lib.stk_setup(8, 0, 1.0, None, ctypes.byref(P)) == -1  # degree out of range
    assert b"degree" in lib.stk_last_error(None)
    assert lib.stk_setup(10, 2, 1.0, None, ctypes.byref(P)) == -1  # not 2 or 3 times a power of two
    assert lib.stk_setup(8, 2, -1.0, None, ctypes.byref(P)) == -1  # viscosity
    assert lib.stk_destroy(None) == 0
    # batched entry points reject empty or NULL arguments before touching a device
    assert lib.stk_smooth_batch(None, 0, None, 0, None, None) == -1
    assert b"smooth_batch" in lib.stk_last_error(None)
    assert lib.stk_solve_batch(None, 0, None, None, ctypes.c_double(1e-8), None) == -1


def test_binding_layout_matches_oracle_numbering():
    from oracle.discretization import Discretization
    from paper_2410_09497_gb300 import layout_sizes

    for n, k in [(2, 1), (6, 3), (64, 3)]:
        d = Discretization(n, k)
        assert layout_sizes(n, k) == (d.n_vel_component, d.n_pressure, d.N)
