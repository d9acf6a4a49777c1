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
    names = set(re.findall(r"\b(rk_[a-z0-9_]+)\s*\(", text))
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


def test_struct_layouts_match_header(tmp_path):
    """The binding's structures have the size and field offsets that a C
    compiler gives the header's (gcc on the host, which uses the same
    layout rules as the device compiler's host side)."""
    import shutil
    import subprocess
    from paper_1501_03358_gb300 import native
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"rk_grid": native.rk_grid, "rk_solve_params": native.rk_solve_params,
               "rk_solve_info": native.rk_solve_info, "rk_prof_entry": native.rk_prof_entry}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rk.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
