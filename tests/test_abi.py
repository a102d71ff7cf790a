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


def test_mesh_sizes_and_parameters_checked_on_the_host():
    """flexi_mesh_init rejects empty meshes, unsupported orders and meshes beyond the
    side-index range before any CUDA call (the coordinate and connectivity buffers are
    not read on these paths, so small placeholders serve)."""
    import numpy as np

    from paper_1910_02858_gb300 import flexi as F

    L = F.lib()
    coords = np.zeros((1, 8, 3))
    conn = np.zeros((1, 6, 3), dtype=np.int32)
    cp, kp = coords.ctypes.data_as(ctypes.c_void_p), conn.ctypes.data_as(ctypes.c_void_p)

    def init(K, **kw):
        p = F.flexi_params(**dict(dict(N=3, Ngeo=1, gamma=1.4, Pr=0.72, mu=1e-3), **kw))
        ctx = ctypes.c_void_p()
        return L.flexi_mesh_init(ctypes.byref(ctx), ctypes.byref(p), K, cp, kp, None)

    assert init(0) == F.FLEXI_EINVAL
    assert init(-3) == F.FLEXI_EINVAL
    assert init(1, N=0) == F.FLEXI_EINVAL
    assert init(1, N=8) == F.FLEXI_EUNSUPPORTED
    assert init(1, Ngeo=4) == F.FLEXI_EINVAL  # Ngeo > N
    assert init(1, node_type=2) == F.FLEXI_EINVAL
    assert init(1, riemann=5) == F.FLEXI_EINVAL
    assert init(1, precision=4) == F.FLEXI_EINVAL
    assert init(1, gamma=1.0) == F.FLEXI_EINVAL
    assert init(1, mu=-1.0) == F.FLEXI_EINVAL
    assert init(1, split_form=1, node_type=0) == F.FLEXI_EUNSUPPORTED  # split form needs Gauss-Lobatto
    assert init(1, lifting=1, precision=2) == F.FLEXI_EUNSUPPORTED  # BR2 on the tensor-core sweeps
    # 6 K side slots must stay below 2^27 (packed side indices)
    assert init((1 << 27) // 6 + 1) == F.FLEXI_EUNSUPPORTED
