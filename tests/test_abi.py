"""The C ABI library loads and exports every entry point include/pinv.h declares.

CPU-only: nothing here launches a kernel or touches a GPU.
"""
import os
import re
import subprocess

import pytest

from paper_2410_06129_gb300 import _lib as L
from paper_2410_06129_gb300 import build as B

HEADER_DIR = os.path.join(B.ROOT, "include")


def _declared():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if fn.endswith(".h"):
            txt = open(os.path.join(HEADER_DIR, fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w \*]*?\b(pinv_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    srcs = B.sources() + [os.path.join(HEADER_DIR, "pinv.h")]
    stale = (not os.path.exists(B.LIB)) or any(os.path.getmtime(s) > os.path.getmtime(B.LIB) for s in srcs)
    if stale:
        B.build()
    return B.LIB


def test_header_declares_entry_points():
    names = _declared()
    assert "pinv_plan_create" in names and "pinv_apply" in names and "pinv_build" in names
    assert set(names) <= set(L.SIGNATURES), "binding lacks a declared symbol"


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pinv_\w+)", out))
    missing = set(_declared()) - exported
    assert not missing, f"not exported: {missing}"


def test_library_loads_without_gpu(lib_path):
    lib = L.load(lib_path)
    for name in _declared():
        assert hasattr(lib, name)
    assert lib.pinv_version() >= 100
    assert lib.pinv_last_error() == b""


def test_invalid_descriptor_rejected_on_host(lib_path):
    """Argument validation happens before any CUDA call."""
    import ctypes as C
    import numpy as np
    lib = L.load(lib_path)
    d, keep = L.make_desc((4, 4), np.zeros((8, 2)))
    d.ndim = 5
    h = C.c_void_p()
    st = lib.pinv_plan_create(C.byref(d), None, C.byref(h))
    assert st == L.ERR_INVALID_ARG
    assert b"ndim" in lib.pinv_last_error()
    d, keep = L.make_desc((4, 4), np.zeros((8, 2)), b0_hz=np.zeros(16), times=np.zeros(8))
    d.times = None
    assert lib.pinv_plan_create(C.byref(d), None, C.byref(h)) == L.ERR_INVALID_ARG
    d, keep = L.make_desc((4, 4), np.zeros((8, 2)), coil_maps=np.ones((2, 16), complex))
    d.coil_maps = None
    assert lib.pinv_plan_create(C.byref(d), None, C.byref(h)) == L.ERR_INVALID_ARG
    d, keep = L.make_desc((4, 4), np.zeros((8, 2)), voxel_index=np.array([0, 3, 99]))
    assert lib.pinv_plan_create(C.byref(d), None, C.byref(h)) == L.ERR_INVALID_ARG
    assert lib.pinv_build(None, None) == L.ERR_INVALID_ARG
    assert lib.pinv_apply(None, None, None, 1, 0, None) == L.ERR_INVALID_ARG
