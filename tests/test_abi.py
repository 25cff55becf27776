"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/rubix.h (no compute calls: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(rubix_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2412_08265_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("rubix_cube_create", "rubix_cube_forward", "rubix_cube_backward", "rubix_cube_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_matches(lib_path):
    from paper_2412_08265_gb300 import capi
    lib = capi.load()
    assert capi.rubix_version().startswith("rubix-gb300")
    for n in declared_symbols():
        assert hasattr(lib, n)
    assert set(capi.exported_symbols()) <= set(declared_symbols())


def test_invalid_arguments_are_reported_without_a_gpu(lib_path):
    """Argument validation happens on the host before any CUDA call."""
    from paper_2412_08265_gb300 import capi
    capi.load()
    h = ctypes.c_void_p()
    rc = capi.load().rubix_cube_create(None, None, 0, ctypes.byref(h))
    assert rc == capi.RUBIX_ERR_INVALID_ARG and h.value is None
    assert b"NULL" in capi.load().rubix_last_error_message()



def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of rubix_ssp_grid, rubix_telescope and rubix_particles
    have the size and field offsets the C compiler gives the header's structs."""
    import ctypes
    import subprocess
    from paper_2412_08265_gb300 import capi
    structs = {"rubix_ssp_grid": capi.rubix_ssp_grid, "rubix_telescope": capi.rubix_telescope,
               "rubix_particles": capi.rubix_particles}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rubix.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    subprocess.check_call(["gcc", "-I", os.path.join(root, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {}
    for l in out:
        if l:
            parts = l.split()
            got[tuple(parts[:-1])] = int(parts[-1])
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_every_entry_point_has_a_binding():
    """The Python binding exposes every function the header declares, by name."""
    from paper_2412_08265_gb300 import capi
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "include", "rubix.h")) as f:
        names = set(re.findall(r"\b(rubix_[a-z0-9_]+)\s*\(", f.read()))
    assert names
    missing = [n for n in sorted(names) if not hasattr(capi, n)]
    assert not missing, missing


def test_missing_library_fails_loudly(tmp_path):
    """Without the CUDA library the binding raises; there is no CPU fallback."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2412_08265_gb300 import capi\n"
            "capi.LIB_PATH = %r\n"
            "try:\n"
            "    capi.rubix_version()\n"
            "except RuntimeError as e:\n"
            "    print('RAISED', e)\n") % (root, str(tmp_path / "absent" / "librubix.so"))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert "RAISED CUDA library not built" in out.stdout, out.stdout + out.stderr
