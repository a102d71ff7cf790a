"""The C-ABI library builds, loads and exports every entry point that
include/flexi.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(flexi_\w+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_02858_gb300 import build as b

    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("flexi_mesh_init", "flexi_rhs", "flexi_rk_step", "flexi_adjoint_step"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1910_02858_gb300 import flexi as F

    assert set(declared_functions()) <= set(F.EXPORTS)


def test_strerror_without_gpu(lib):
    lib.flexi_strerror.restype = ctypes.c_char_p
    assert lib.flexi_strerror(-4).decode().startswith("invalid mesh")
    assert lib.flexi_strerror(0).decode() == "ok"


def test_invalid_arguments_rejected_before_device_work(lib):
    """Null pointers and out-of-range sizes fail on the host with FLEXI_EINVAL."""
    lib.flexi_mesh_init.restype = ctypes.c_int
    assert lib.flexi_mesh_init(None, None, 0, None, None, None) == -1
    lib.flexi_rhs.restype = ctypes.c_int
    lib.flexi_rhs.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
    assert lib.flexi_rhs(None, None, None, 0.0, None) == -1
