"""CPU checks of the boundary: the library builds and loads, and it exports
every function include/linview.h declares (no compute calls: no GPU here)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "linview.h")).read()
    return sorted(set(re.findall(r"\b(linview_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    import ctypes
    from paper_1403_6968_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    names = _declared()
    assert "linview_create_program" in names and "linview_apply_delta" in names
    for name in names:
        assert hasattr(lib, name), name
    # the binding declares a signature for every exported function
    assert set(names) == set(_lib.EXPORTED)


def test_errors_without_device_are_status_codes():
    import ctypes as C
    from paper_1403_6968_gb300 import _lib
    lib = _lib.load()
    d = _lib.ProgramDesc()
    d.kind, d.precision, d.n, d.k, d.r_max = _lib.POWER, _lib.F32, 4, 2, 1
    h = C.c_void_p()
    a = (C.c_float * 16)()
    ptrs = (C.c_void_p * 1)(C.cast(a, C.c_void_p))
    lds = (C.c_int64 * 1)(4)
    st = lib.linview_create_program(C.byref(d), ptrs, lds, 0, None, C.byref(h))
    # no GPU in this container: EDEVICE; on a GPU machine: OK
    assert st in (_lib.OK, _lib.EDEVICE)
    if st == _lib.OK:
        lib.linview_destroy(h)
    else:
        assert b"device" in lib.linview_last_error().lower()
    d.k = 3  # not a power of two: rejected before any device work
    assert lib.linview_create_program(None, ptrs, lds, 0, None, C.byref(h)) == _lib.EINVAL


def test_python_binding_fails_loudly_without_library(tmp_path):
    import pytest
    from paper_1403_6968_gb300 import _lib
    with pytest.raises(ImportError):
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "missing.so"))
        finally:
            _lib._lib = None


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C layout (sizes and
    field offsets, from a C program compiled against include/linview.h)."""
    import ctypes as C
    import os
    import shutil
    import subprocess
    import pytest
    from paper_1403_6968_gb300 import _lib
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"linview_program_desc": _lib.ProgramDesc, "linview_completion": _lib.Completion,
               "linview_server_stats": _lib.ServerStats}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "linview.h"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True,
                             text=True).stdout.splitlines():
        cname, field, val = ln.split()
        got[(cname, field)] = int(val)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
