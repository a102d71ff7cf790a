"""RK steps through the small-mesh FP64 kernels against the FP64 oracle.

A mesh with fewer elements than SMs at N = 3 runs each RK stage as the lifting/volume
kernel plus one fused kernel that computes the face fluxes itself and applies the surface
integral, the RK update and the new face states (two CTAs per element on Gauss-Lobatto
nodes), with the face states in rotating buffers.  The right-hand-side parity tests go
through the separate face and surface kernels, so these cases check the fused path for
every numerical flux, boundary kind, split form and the source term: five steps, 1e-12
relative L2 per conserved variable, the bar of the other state tests.
"""
import numpy as np
import pytest
import torch

import workloads as wl

from test_gpu_bc import _pair
from test_gpu_parity import DEV, _oracle, _solver, per_var_rel

pytestmark = pytest.mark.gpu

BOX = dict(lo=(-1,) * 3, hi=(1,) * 3, periodic=(False,) * 3)

BC_CASES = [
    # (name, mesh kwargs, solver kwargs, boundary kinds): slip walls, inflow (exact state) and outflow
    ("walls_lg_hllc", dict(BOX, nelem=(2, 2, 3), Ngeo=3, mapping="sine", reorient_seed=11, bc_ids=[2] * 6),
     dict(N=3, Ngeo=3, riemann=1), {2: 2}),
    ("walls_lgl_roe", dict(BOX, nelem=(3, 2, 2), Ngeo=3, mapping="sine", reorient_seed=12, bc_ids=[2] * 6),
     dict(N=3, Ngeo=3, node_type=1, riemann=0, mu=1 / 400.0), {2: 2}),
    ("in_out_lg_rusanov", dict(BOX, nelem=(3, 2, 2), periodic=(False, True, True), reorient_seed=13,
                               bc_ids=[0, 1, 0, 0, 0, 0]), dict(N=3, riemann=3, bc_exact=1), {1: 1}),
    ("in_out_lgl_rusanov", dict(BOX, nelem=(2, 3, 2), periodic=(False, True, True), reorient_seed=14,
                                bc_ids=[0, 1, 0, 0, 0, 0]), dict(N=3, node_type=1, riemann=3, bc_exact=1), {1: 1}),
]


@pytest.mark.parametrize("name,mk,sk,kinds", BC_CASES, ids=[c[0] for c in BC_CASES])
def test_fused_steps_with_boundaries(name, mk, sk, kinds):
    mesh = wl.box_mesh(**mk)
    s, dg = _pair(dict(sk, precision=0), mesh, kinds)
    U0 = wl.perturbed(np.pi * mesh.node_coords(3, sk.get("node_type", 0)), seed=21)
    U = torch.tensor(U0, device=DEV)
    s.run(U, 5, 5e-4)
    ref = dg.run(torch.tensor(U0), 5, 5e-4)
    s.close()
    err = per_var_rel(U, ref)
    assert err < 1e-12, err


PERIODIC_CASES = [
    # smoothed Roe with the kinetic-energy-preserving split form, the entropy-conservative
    # flux with its split form (Gauss-Lobatto: two CTAs per element), HLLC on Gauss nodes
    ("kep_lgl_roesmooth", dict(nelem=(3, 3, 2), reorient_seed=15), dict(N=3, node_type=1, riemann=2,
                                                                       split_form=1, mu=1 / 400.0)),
    ("ec_lgl_ec", dict(nelem=(2, 3, 3), reorient_seed=16), dict(N=3, node_type=1, riemann=4, split_form=2)),
    ("lg_hllc", dict(nelem=(3, 2, 3), reorient_seed=17), dict(N=3, riemann=1)),
]


@pytest.mark.parametrize("name,mk,sk", PERIODIC_CASES, ids=[c[0] for c in PERIODIC_CASES])
def test_fused_steps_periodic(name, mk, sk):
    mesh = wl.box_mesh(Ngeo=1, **mk)
    sk = dict(sk, precision=0)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = wl.perturbed(mesh.node_coords(3, sk.get("node_type", 0)), seed=22)
    U = torch.tensor(U0, device=DEV)
    s.run(U, 5, 1e-3)
    ref = dg.run(torch.tensor(U0), 5, 1e-3)
    s.close()
    err = per_var_rel(U, ref)
    assert err < 1e-12, err


@pytest.mark.parametrize("nt", [0, 1], ids=["lg", "lgl"])
def test_fused_steps_manufactured_source(nt):
    """Curved mesh, exact-state boundaries of the time-dependent manufactured solution and
    its source term (the time-dependent operator takes the eager path of flexi_rk_run)."""
    mesh = wl.box_mesh((2, 3, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=3, mapping="sine", periodic=(False, True, False))
    sk = dict(N=3, Ngeo=3, node_type=nt, riemann=1, bc_exact=2, source=True, precision=0)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = wl.manufactured(mesh.node_coords(3, nt), 0.1)
    U = torch.tensor(U0, device=DEV)
    s.run(U, 5, 1e-3, t0=0.1)
    ref = dg.run(torch.tensor(U0), 5, 1e-3, t0=0.1)
    s.close()
    err = per_var_rel(U, ref)
    assert err < 1e-12, err
