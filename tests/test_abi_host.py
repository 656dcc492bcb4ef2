"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function that include/fem.h declares, and its
argument checks reject bad calls before any CUDA work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1501_04784_gb300 import _build, abi
    _build.build()
    return abi.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fem_[a-z_A-Z0-9]+)\s*\(", src)))


def test_exports_every_declared_function(lib):
    from paper_1501_04784_gb300 import abi
    names = declared_functions()
    assert len(names) >= 15
    assert set(names) == set(abi.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_defaults(lib):
    from paper_1501_04784_gb300 import abi
    for code, name in abi.STATUS.items():
        assert lib.fem_status_str(code).decode() == name
    o = abi.fem_options()
    lib.fem_options_default(ctypes.byref(o))
    assert o.valence_threshold == 8 and o.locality_order == 1 and o.mem_budget_bytes == 0


def test_argument_checks_fail_before_cuda(lib):
    from paper_1501_04784_gb300 import abi
    h = ctypes.c_void_p()
    st = lib.fem_mesh_create(ctypes.byref(h), 8, 10, 1, None, None, 0, None, None)
    assert st == 1  # FEM_ERR_ARG
    assert b"E must be" in lib.fem_last_error()
    st = lib.fem_mesh_create(ctypes.byref(h), 7, 10, 1, ctypes.c_void_p(16), None, 0, None, None)
    assert st == 1 and b"element type" in lib.fem_last_error()
    st = lib.fem_mesh_create(ctypes.byref(h), 8, 0, 1, ctypes.c_void_p(16), None, 0, None, None)
    assert st == 1 and b"sizes" in lib.fem_last_error()
    st = lib.fem_mesh_create(ctypes.byref(h), 8, 10, 1, ctypes.c_void_p(18), None, 0, None, None)
    assert st == 1 and b"aligned" in lib.fem_last_error()
    assert lib.fem_build_K(None, 0, None, 1, None, 1, None, None) == 1
    assert lib.fem_pattern(None, None, None) == 1
    info = abi.fem_info()
    assert lib.fem_mesh_info(None, ctypes.byref(info)) == 1
    lib.fem_mesh_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1501_04784_gb300 import _build, abi
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(abi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        abi.load()


def test_struct_mirrors_match_the_header(tmp_path):
    """The binding's ctypes mirrors of fem_options, fem_info and fem_tuning have
    the C structs' size and every field's offset (a C program compiled against
    include/fem.h prints them)."""
    import shutil
    import subprocess
    from paper_1501_04784_gb300 import abi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [("fem_options", abi.fem_options), ("fem_info", abi.fem_info), ("fem_tuning", abi.fem_tuning)]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fem.h"', "int main(void) {"]
    for cname, py in structs:
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for cname, py in structs:
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
