"""flexi_reduce_noalloc: the global reductions without any device allocation.

Callers that cannot allocate device memory when they need the conserved totals,
kinetic energy or the stable time step (for instance because their own memory
manager owns the device, or because cudaMalloc/cudaFree would synchronise the
device in the middle of a time loop) use this entry point; it keeps its partial
sums in a fixed array of the library's static device memory.  The test checks
it through the C ABI against flexi_reduce, which uses the context's buffer, on
two calls in a row (the static array keeps the previous call's contents), with
and without U_t, in FP64 and FP32, and that meshes above the stated maximum are
rejected.  This file is collected last on purpose.
"""
import pytest
import torch

import workloads as wl

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _solver(mesh, **kw):
    from paper_1910_02858_gb300 import Solver, SolverConfig
    from paper_1910_02858_gb300 import build as b

    b.build()
    return Solver(SolverConfig(**kw), mesh.coords, mesh.conn, device=DEV)


def _compare(ref, got):
    for q in range(8):
        scale = max(1.0, abs(ref[q]))
        assert abs(got[q] - ref[q]) <= 1e-12 * scale, (q, ref[q], got[q])


@pytest.mark.parametrize("nel,N,precision", [(16, 7, 0), (8, 5, 1), (5, 3, 0)])
def test_noalloc_matches_reduce_twice(nel, N, precision):
    from paper_1910_02858_gb300 import flexi as F

    mesh = wl.box_mesh((nel, nel, nel), Ngeo=1, reorient_seed=nel)
    s = _solver(mesh, N=N, riemann=F.RIEMANN_HLLC, precision=precision)
    U = torch.tensor(wl.taylor_green(mesh.node_coords(N, 0)), device=DEV, dtype=s.dtype)
    Ut = s.rhs(U)
    stream = torch.cuda.current_stream()
    for Ut_arg in (None, Ut, None):  # consecutive calls reuse the static array
        ref, rc = F.flexi_reduce(s.ctx, U, Ut_arg, 0.9, stream)
        got, code = F.flexi_reduce_noalloc(s.ctx, U, Ut_arg, 0.9, stream)
        assert code == F.FLEXI_OK
        _compare(ref, got)
    s.close()


def test_noalloc_rejects_meshes_above_the_limit():
    from paper_1910_02858_gb300 import flexi as F

    n = 41  # 41^3 = 68921 > 65536 elements
    assert n ** 3 > F.NOALLOC_MAX_ELEMENTS
    mesh = wl.box_mesh((n, n, n), Ngeo=1)
    s = _solver(mesh, N=1, riemann=F.RIEMANN_HLLC)
    U = torch.tensor(wl.taylor_green(mesh.node_coords(1, 0)), device=DEV)
    _, code = F.flexi_reduce_noalloc(s.ctx, U, None, 0.9, torch.cuda.current_stream())
    assert code == F.FLEXI_EINVAL
    vals, rc = F.flexi_reduce(s.ctx, U, None, 0.9, torch.cuda.current_stream())  # the allocating path still works
    assert rc == F.FLEXI_OK and vals[0] > 0
    s.close()
