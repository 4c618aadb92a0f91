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
    # an in-place batched solve (x[i] == b[i]) is refused before the problem is
    # touched (the handle here is a host buffer that no call may use)
    dummy = ctypes.create_string_buffer(256)
    probs = (ctypes.c_void_p * 1)(ctypes.addressof(dummy))
    same = (ctypes.c_void_p * 1)(4096)
    lib.stk_solve_batch.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
    assert lib.stk_solve_batch(probs, 1, same, same, ctypes.c_double(1e-8), None) == -1
    assert b"alias" in lib.stk_last_error(None)


def test_binding_layout_matches_oracle_numbering():
    from oracle.discretization import Discretization
    from paper_2410_09497_gb300 import layout_sizes

    for n, k in [(2, 1), (6, 3), (64, 3)]:
        d = Discretization(n, k)
        assert layout_sizes(n, k) == (d.n_vel_component, d.n_pressure, d.N)


def _build_c_program(tmp_path):
    import shutil
    import subprocess

    from paper_2410_09497_gb300 import build

    lib = build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "c_abi_check")
    libdir = os.path.dirname(lib)
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_check.c"), "-o", exe, "-L", libdir, "-lstokesmg",
           "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_against_the_header(tmp_path):
    """The header compiles as strict C99 and a C program linked to the library
    gets status codes and messages back without a GPU."""
    import subprocess

    exe = _build_c_program(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and "c abi ok" in r.stdout, (r.returncode, r.stdout, r.stderr)


@pytest.mark.gpu
def test_c_program_sets_up_a_problem(tmp_path):
    import subprocess

    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = _build_c_program(tmp_path)
    r = subprocess.run([exe, "gpu"], capture_output=True, text=True)
    assert r.returncode == 0 and "layout n=4" in r.stdout, (r.returncode, r.stdout, r.stderr)


def test_every_entry_point_cites_its_passage():
    """Each declaration in include/*.h is preceded by a comment that cites the
    passage of the paper defining the operation, or says it has none."""
    missing = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        decls = re.finditer(r"/\*((?:(?!\*/).)*)\*/\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(stk_[A-Za-z0-9_]+)\s*\(", text, flags=re.S)
        found = {}
        for m in decls:
            found[m.group(2)] = bool(re.search(r"Sec\.|eq\.|Algorithm|Table|no counterpart", m.group(1)))
        missing += [n for n, ok in found.items() if not ok]
        missing += [n for n in declared_symbols() if n not in found and os.path.basename(h) == "stokesmg.h"]
    assert not missing, missing
