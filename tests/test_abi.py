"""The C-ABI library builds, loads and exports every entry point that
include/ppe.h declares; host-only calls work without a GPU."""
import os
import re

import pytest

from paper_2103_01874_gb300 import build, ppe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*[\w\s\*]*?\b(ppe_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ppe.lib()


def test_header_declares_the_api():
    names = declared_functions()
    for want in ("ppe_plan", "ppe_rhs", "ppe_solve", "ppe_correct", "ppe_project", "ppe_destroy", "ppe_strerror"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    assert declared_functions() <= set(ppe.SIGNATURES)


def test_host_only_calls(lib):
    assert ppe.size_supported(256, 256, 256)
    assert ppe.size_supported(384, 256, 384)
    assert ppe.size_supported(18, 27, 54)
    assert not ppe.size_supported(250, 8, 8)
    assert not ppe.size_supported(9, 8, 8)     # odd nx
    assert not ppe.size_supported(4, 8, 8)     # below 8
    assert not ppe.size_supported(2048, 8, 8)  # above the maximum
    for code in range(8):
        assert lib.ppe_strerror(code)
    g = ppe.Grid(256, 256, 256, 1.0, 1.0, 1.0)
    o64 = ppe.Options(ppe.FP64, 0, 1e-10, 4, 1e-12)
    o32 = ppe.Options(ppe.FP32_REFINE, 0, 1e-10, 4, 1e-12)
    import ctypes
    b64 = lib.ppe_workspace_bytes(ctypes.byref(g), ctypes.byref(o64))
    b32 = lib.ppe_workspace_bytes(ctypes.byref(g), ctypes.byref(o32))
    assert b64 > 16 * 129 * 256 * 256 and b32 > 8 * 129 * 256 * 256


def test_null_arguments_rejected(lib):
    import ctypes
    assert lib.ppe_plan(None, None, None, None) == 1
    assert lib.ppe_solve(None, None, None) == 1
    assert lib.ppe_project(None, None) == 1
    lib.ppe_destroy(None)
    h = ctypes.c_void_p()
    g = ppe.Grid(250, 8, 8, 1.0, 1.0, 1.0)
    assert lib.ppe_plan(ctypes.byref(h), ctypes.byref(g), None, None) == 2
    g = ppe.Grid(8, 8, 8, -1.0, 1.0, 1.0)
    assert lib.ppe_plan(ctypes.byref(h), ctypes.byref(g), None, None) == 1
