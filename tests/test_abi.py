"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/rk.h declares (no GPU compute here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "rk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(rk_[a-z_]+)\s*\(", text))
    return sorted(n for n in names if not n.endswith("_fn"))


@pytest.fixture(scope="module")
def lib():
    from paper_1501_03358_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("rk_create_problem", "rk_set_recycle", "rk_solve", "rk_get_recycle"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_1501_03358_gb300 import native
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(declared_symbols()) == set(native.EXPORTS)


def test_version_and_error_without_gpu(lib):
    lib.rk_version.restype = ctypes.c_char_p
    lib.rk_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.rk_version()
    assert isinstance(lib.rk_last_error(), bytes)


def test_struct_layouts_match_header():
    from paper_1501_03358_gb300 import native
    assert ctypes.sizeof(native.rk_grid) == 16
    assert ctypes.sizeof(native.rk_solve_params) == 8 + 8 * 4
    assert ctypes.sizeof(native.rk_solve_info) == 6 * 4 + 3 * 8
