"""Boundary kinds on the GPU (flexi_set_bc: exact state, outflow, slip wall)
through the C ABI against the oracle's boundary kinds.

Right-hand sides use the rounding-sensitivity tolerance of test_gpu_parity (1-ulp
noise on the state and on the mesh coordinates, 20 sigma; FP32 scaled by 2^29);
states after time steps 1e-12 relative L2 per conserved variable (FP64)."""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import equations as eq
from oracle.dgsem import DGSEM, HLLC, ROE, RUSANOV, Params

from test_gpu_parity import DEV, per_var_rel, rhs_parity_ok, rounding_sensitivity

pytestmark = pytest.mark.gpu

RIEM = {0: ROE, 1: HLLC, 3: RUSANOV}


def _pair(sk, mesh, kinds):
    from paper_1910_02858_gb300 import Solver, SolverConfig

    s = Solver(SolverConfig(**sk), mesh.coords, mesh.conn, device=DEV)
    for bc_id, kind in kinds.items():
        s.set_bc(bc_id, kind)
    dg = DGSEM(Params(N=sk["N"], node_type=sk.get("node_type", 0), riemann=RIEM[sk.get("riemann", 0)],
                      mu=sk.get("mu", 1 / 1600.0), bc_exact=sk.get("bc_exact", 0), bc_kinds=dict(kinds)),
               mesh.coords, mesh.conn)
    return s, dg


CASES = [
    # (name, mesh kwargs, solver kwargs, boundary kinds)
    ("slip_box_lg_N3_hllc", dict(nelem=(2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=3, mapping="sine",
                                 periodic=(False,) * 3, reorient_seed=1, bc_ids=[2] * 6),
     dict(N=3, Ngeo=3, riemann=1), {2: 2}),
    ("slip_box_lgl_N5_roe", dict(nelem=(2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=2, mapping="sine",
                                 periodic=(False,) * 3, reorient_seed=2, bc_ids=[2] * 6),
     dict(N=5, Ngeo=2, node_type=1, riemann=0, mu=1 / 400.0), {2: 2}),
    ("in_out_lg_N7_rusanov", dict(nelem=(3, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, periodic=(False, True, True),
                                  reorient_seed=3, bc_ids=[0, 1, 0, 0, 0, 0]),
     dict(N=7, riemann=3, bc_exact=1), {1: 1}),
    ("mixed_lg_N4_hllc", dict(nelem=(2, 3, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=4, mapping="sine",
                              periodic=(False,) * 3, reorient_seed=4, bc_ids=[0, 1, 2, 2, 2, 2]),
     dict(N=4, Ngeo=4, riemann=1, bc_exact=1), {1: 1, 2: 2}),
]


@pytest.mark.parametrize("name,mk,sk,kinds", CASES, ids=[c[0] for c in CASES])
def test_bc_rhs_parity_fp64(name, mk, sk, kinds):
    mesh = wl.box_mesh(**mk)
    s, dg = _pair(dict(sk, precision=0), mesh, kinds)
    U0 = wl.perturbed(np.pi * mesh.node_coords(sk["N"], sk.get("node_type", 0)), seed=7)
    Ut = s.rhs(torch.tensor(U0, device=DEV), 0.2)
    ok, d, tol = rhs_parity_ok(Ut, dg, torch.tensor(U0), 0.2, mesh)
    s.close()
    assert ok, (d, tol)


def test_bc_rhs_parity_fp32():
    name, mk, sk, kinds = CASES[3]
    mesh = wl.box_mesh(**mk)
    s, dg = _pair(dict(sk, precision=1), mesh, kinds)
    U0 = wl.perturbed(np.pi * mesh.node_coords(sk["N"], 0), seed=7)
    Ut = s.rhs(torch.tensor(U0, device=DEV, dtype=torch.float32), 0.0)
    ref, parts = dg.rhs(torch.tensor(U0), 0.0, parts=True)
    scale = (ref.abs() + (parts["vol"] / dg.geo.J.unsqueeze(1)).abs()).transpose(0, 1).reshape(5, -1).norm(dim=1)
    sig = rounding_sensitivity(dg, torch.tensor(U0), 0.0, mesh=mesh) * 2.0 ** 29
    d = (Ut.double().cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    tol = torch.maximum(3e-6 * scale, 20 * sig)
    s.close()
    assert bool((d <= tol).all()), (d.tolist(), tol.tolist())


def test_bc_rk_steps_match_oracle():
    name, mk, sk, kinds = CASES[3]
    mesh = wl.box_mesh(**mk)
    s, dg = _pair(sk, mesh, kinds)
    U0 = wl.perturbed(np.pi * mesh.node_coords(sk["N"], 0), seed=7)
    U = torch.tensor(U0, device=DEV)
    s.run(U, 20, 5e-4)
    Ur = dg.run(torch.tensor(U0), 20, 5e-4)
    err = per_var_rel(U, Ur)
    s.close()
    assert err < 1e-12, err


def test_closed_box_conserves_mass_100_steps():
    """N = 7 curved box closed by slip walls: total mass stays constant over 100
    steps (the mirror state makes the walls' mass flux vanish)."""
    N = 7
    mesh = wl.box_mesh((3, 3, 3), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3,
                       reorient_seed=5, bc_ids=[2] * 6)
    s, _ = _pair(dict(N=N, Ngeo=N, riemann=1, mu=1 / 400.0), mesh, {2: 2})
    U = torch.tensor(wl.perturbed(np.pi * mesh.node_coords(N, 0), seed=8), device=DEV)
    r0 = s.reduce(U)
    s.run(U, 100, 0.5 * r0["dt_max"])
    r1 = s.reduce(U)
    assert abs(r1["mass"] - r0["mass"]) < 1e-12 * abs(r0["mass"])
    s.close()


def test_set_bc_errors():
    from paper_1910_02858_gb300 import flexi as F

    mesh = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, periodic=(False,) * 3, bc_ids=[2] * 6)
    s, _ = _pair(dict(N=2), mesh, {})
    for bc_id, kind in ((7, F.BC_OUTFLOW), (2, 3), (2, -1)):  # no side with id 7; unknown kinds
        with pytest.raises(F.FlexiError) as ei:
            s.set_bc(bc_id, kind)
        assert ei.value.code == F.FLEXI_EINVAL
    s.set_bc(2, F.BC_SLIP_WALL)
    s.close()
