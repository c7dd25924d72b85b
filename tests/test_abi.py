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


def test_workspace_counts_the_fp32_first_solve_pressure(lib):
    """ppe_project keeps the first solve's p in FP32 (4 B per cell more
    workspace) exactly where the inverse transforms' scaling 1/((nx/2) nz) is a
    power of two and nx/2 has a register-staged length (16 .. 256), in the FP32
    form with at least one sweep; the bench's byte accounting makes the same
    call."""
    import ctypes
    import bench

    def ws(shape, precision, sweeps):
        g = ppe.Grid(*shape, 1.0, 1.0, 1.0)
        o = ppe.Options(precision, 0, 1e-10, sweeps, 1e-12)
        return lib.ppe_workspace_bytes(ctypes.byref(g), ctypes.byref(o))

    cases = [((256, 256, 256), True), ((64, 48, 32), True), ((512, 64, 64), True), ((32, 8, 16), True),
             ((1024, 8, 8), False),   # nx/2 = 512: no compiled register-staged length
             ((384, 256, 384), False),  # nx/2 = 192 not a power of two
             ((256, 64, 48), False),  # (nx/2) nz = 6144 not a power of two
             ((24, 16, 16), False)]   # nx/2 = 12 below 16
    for shape, eligible in cases:
        n = shape[0] * shape[1] * shape[2]
        extra = ws(shape, ppe.FP32_REFINE, 4) - ws(shape, ppe.FP32_REFINE, 0)
        assert extra == (4 * n if eligible else 0), (shape, extra)
        assert ws(shape, ppe.FP64, 4) == ws(shape, ppe.FP64, 0)
        old = (bench.NX, bench.NY, bench.NZ)
        try:
            bench.NX, bench.NY, bench.NZ = shape
            assert bench.p0_fp32() == eligible, shape
        finally:
            bench.NX, bench.NY, bench.NZ = old
