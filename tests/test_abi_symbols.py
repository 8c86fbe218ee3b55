"""The C-ABI library loads without a GPU and exports every entry point that
include/*.h declares (no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(dd\w*)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    import paper_2311_08757_gb300 as pkg
    from paper_2311_08757_gb300 import _build
    if not os.path.exists(pkg.lib_path()):
        _build.build()
    return pkg.lib_path()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("dd_setup", "dd_cell_eigenpair", "dd_coarse_build", "dd_pcg_solve",
                 "dd_inverse_iterate", "dd_eigenpair", "dd_destroy", "dd_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    import paper_2311_08757_gb300 as dd
    assert dd.status_string(dd.DD_OK) == "DD_OK"
    assert dd.status_string(dd.DD_ENOTSPD) == "DD_ENOTSPD"
    assert dd.status_string(12345) == "DD_UNKNOWN"


def test_binding_signatures_cover_header():
    import paper_2311_08757_gb300 as dd
    assert set(declared_symbols()) <= set(dd._SIGS)


@pytest.mark.parametrize("struct", ["dd_grid", "dd_info"])
def test_binding_structs_match_the_header(struct, tmp_path):
    """The ctypes structures of the binding have the header's size and field offsets (read
    from a C program compiled against include/ddeig.h)."""
    import shutil
    import subprocess
    import paper_2311_08757_gb300 as pkg
    if shutil.which("gcc") is None:
        pytest.skip("gcc not found")
    cls = getattr(pkg, struct)
    lines = [f'printf("%zu\\n", sizeof({struct}));']
    lines += [f'printf("%zu\\n", offsetof({struct}, {name}));' for name, _ in cls._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"ddeig.h\"\nint main(void) {\n  "
                   + "\n  ".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(cls)] + [getattr(cls, name).offset for name, _ in cls._fields_]
    assert got == want
