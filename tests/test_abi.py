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


def test_struct_layout_matches_header(lib):
    # sizes of the ABI structs as a C compiler lays them out
    assert ctypes.sizeof(lib.hj_grid) == 4 + 4 + 32 + 32 + 32 + 4 + 4
    assert ctypes.sizeof(lib.hj_method) == 4 + 4 + 64 + 4 + 4 + 8 + 8
    assert ctypes.sizeof(lib.hj_stats) == 6 * 8
