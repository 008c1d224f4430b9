"""Host-side checks of the C ABI library (no GPU needed): it builds for
sm_103a, loads, exports every function include/hj.h declares, and rejects
bad arguments without touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_11542_gb300 import build, _lib
    build.build()
    return _lib


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:hj_status|void|const char\*)\s+(hj_\w+)\s*\(", text, re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert {"hj_solve", "hj_rk3_step", "hj_step_bound", "hj_term", "hj_upwind"} <= declared
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in sorted(declared):
        assert hasattr(so, name), name
    assert declared == set(lib.EXPORTS)


def test_status_strings_and_version(lib):
    assert lib.hj_status_str(lib.HJ_OK) == "ok"
    assert lib.hj_status_str(lib.HJ_EINVAL) == "invalid argument"
    assert lib.hj_status_str(99) == "unknown status"
    assert "sm_103a" in lib.hj_version()


def test_null_context_is_rejected(lib):
    L = lib.load()
    g = lib.make_grid(type("G", (), {"n": (8, 8), "lo": (0, 0), "hi": (1, 1), "periodic": ()}))
    m = lib.make_method()
    assert L.hj_term(None, ctypes.byref(g), ctypes.byref(m), lib.HJ_F64, None, None) == lib.HJ_EINVAL
    out = ctypes.c_void_p()
    assert L.hj_ctx_create(0, None, None) == lib.HJ_EINVAL


def test_struct_layout_matches_header(lib, tmp_path):
    # sizes and field offsets of the ABI structs as the C compiler lays them
    # out from include/hj.h, against the ctypes mirrors
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = {"hj_grid": lib.hj_grid, "hj_method": lib.hj_method, "hj_problem": lib.hj_problem,
               "hj_stats": lib.hj_stats, "hj_server_info": lib.hj_server_info, "hj_shape": lib.hj_shape}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hj.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got["%s.%s" % (name, field)]) == getattr(cls, field).offset, (name, field)
