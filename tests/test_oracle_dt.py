"""Pins of the oracle's time-step limit (Sec. 3.4, Eqs. CFLCondition and DFLCondition).

The paper bounds the step by CFL * Delta x / (lambda^c (2N+1)) for the convective
part and by CFL_d * Delta x^2 / (lambda^v (2N+1)) for the diffusive part, with
lambda^v the largest eigenvalue of the diffusion matrix, evaluated for each
reference direction (the element size entering through the mapping) and the
smaller of the two used.  Reading: gamma_RK = 1; the directional rates are summed.

On an affine Cartesian element of widths h_l with a constant state this gives, in
closed form,

    dt_c = CFL   / ((2N+1) * sum_l (|u_l| + c) / h_l)
    dt_v = CFL_d / ((2N+1) * lambda^v * sum_l 1 / h_l^2)

The pins below use hand-evaluated numbers of these expressions on an anisotropic
box (h = 1, 2, 4), so that a dropped 1/J, a swapped direction, a missing square on
h, or a wrong (2N+1) factor changes the result, plus the scaling laws in h and N,
invariance under element reorientation, and lambda^v computed independently as an
eigenvalue of the diffusion matrix of the oracle's own viscous flux.
"""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import equations as eq
from oracle.dgsem import DGSEM, HLLC, Params

GAMMA, PR = 1.4, 0.72


def _dg(N, mu, nelem=(2, 2, 2), hi=(2.0, 4.0, 8.0), node_type=0, reorient_seed=None):
    mesh = wl.box_mesh(nelem, lo=(0.0, 0.0, 0.0), hi=hi, Ngeo=1, reorient_seed=reorient_seed)
    dg = DGSEM(Params(N=N, node_type=node_type, riemann=HLLC, mu=mu, gamma=GAMMA, Pr=PR), mesh.coords, mesh.conn)
    return dg, mesh


def _constant_state(mesh, N, node_type, vel=(0.5, -0.25, 0.0), c=1.0, rho=1.0):
    # p from the sound speed: c^2 = gamma p / rho
    p = rho * c * c / GAMMA
    return torch.tensor(wl.freestream(mesh.node_coords(N, node_type), rho=rho, vel=vel, p=p, gamma=GAMMA))


@pytest.mark.parametrize("node_type", [0, 1])
@pytest.mark.parametrize("seed", [None, 5])
def test_convective_limit_hand_value(node_type, seed):
    """N = 3, h = (1, 2, 4), u = (0.5, -0.25, 0), c = 1, CFL = 0.9:
    sum (|u_l| + c)/h_l = 1.5/1 + 1.25/2 + 1/4 = 2.375, dt = 0.9 / (7 * 2.375)."""
    dg, mesh = _dg(3, mu=1e-9, node_type=node_type, reorient_seed=seed)
    U = _constant_state(mesh, 3, node_type)
    expect = 0.9 / 16.625  # = 0.054135338345864...
    assert abs(dg.dt_max(U, 0.9, 0.9) - expect) < 1e-13 * expect
    # CFL enters linearly
    assert abs(dg.dt_max(U, 0.45, 0.45) - 0.5 * expect) < 1e-13 * expect


@pytest.mark.parametrize("seed", [None, 3])
def test_viscous_limit_hand_value(seed):
    """N = 3, h = (1, 2, 4), mu = 1, rho = 1: lambda^v = (gamma/Pr) mu/rho = 1.4/0.72,
    sum 1/h_l^2 = 1 + 1/4 + 1/16 = 1.3125, dt = 0.9 / (7 * (1.4/0.72) * 1.3125)."""
    dg, mesh = _dg(3, mu=1.0, reorient_seed=seed)
    U = _constant_state(mesh, 3, 0)
    expect_v = 0.9 / (7.0 * (1.4 / 0.72) * 1.3125)  # = 0.050379...
    assert 0.0503 < expect_v < 0.0504
    assert expect_v < 0.9 / 16.625  # the diffusive bound is the smaller one here
    assert abs(dg.dt_max(U, 0.9, 0.9) - expect_v) < 1e-13 * expect_v


def test_scaling_in_h_and_N():
    """Halving every element width halves the convective limit and quarters the
    diffusive one; going from N = 1 to N = 3 divides both by 7/3."""
    Uc = lambda dg, mesh, N: _constant_state(mesh, N, 0)
    dg1, m1 = _dg(3, mu=1e-9)
    dg2, m2 = _dg(3, mu=1e-9, nelem=(4, 4, 4))
    assert abs(dg2.dt_max(Uc(dg2, m2, 3)) / dg1.dt_max(Uc(dg1, m1, 3)) - 0.5) < 1e-13
    dv1, n1 = _dg(3, mu=1.0)
    dv2, n2 = _dg(3, mu=1.0, nelem=(4, 4, 4))
    assert abs(dv2.dt_max(Uc(dv2, n2, 3)) / dv1.dt_max(Uc(dv1, n1, 3)) - 0.25) < 1e-13
    da, ma = _dg(1, mu=1e-9)
    db, mb = _dg(3, mu=1e-9)
    assert abs(da.dt_max(Uc(da, ma, 1)) / db.dt_max(Uc(db, mb, 3)) - 7.0 / 3.0) < 1e-13


def test_limit_taken_at_the_fastest_node():
    """A non-constant state: the limit is set by the largest local rate, so a state
    whose speed is raised in one element only gives that element's closed form."""
    dg, mesh = _dg(2, mu=1e-9)
    x = mesh.node_coords(2, 0)
    U = _constant_state(mesh, 2, 0).clone()
    # element 5 moves at u = (3, 0, 0): rates (3+1)/1 + 1/2 + 1/4 = 4.75
    U[5, 1] = 3.0 * U[5, 0]
    U[5, 4] = U[5, 4] + 0.5 * 9.0 * U[5, 0] - 0.5 * (0.25 + 0.0625) * U[5, 0]
    U[5, 2] = 0.0
    expect = 0.9 / (5.0 * 4.75)
    assert abs(dg.dt_max(U, 0.9, 0.9) - expect) < 1e-13 * expect
    del x


@pytest.mark.parametrize("Pr,ratio", [(0.72, 1.4 / 0.72), (2.0, 4.0 / 3.0)])
def test_diffusion_matrix_largest_eigenvalue(Pr, ratio):
    """lambda^v is the largest eigenvalue of the 1-D diffusion matrix B with
    F^v_1 = B dU/dx1 (Eq. DFLCondition).  B is formed here by differentiating the
    oracle's viscous flux (itself pinned against closed forms) through the chain
    rule W_x = (dW/dU) U_x, and its spectrum computed numerically; the largest
    eigenvalue is max(4/3, gamma/Pr) mu/rho, the value dt_max uses."""
    gas = eq.Gas(GAMMA, Pr, 0.37)
    U0 = eq.cons(torch.tensor([1.7, 0.3, -0.2, 0.1, 2.1], dtype=torch.float64), gas)
    dWdU = torch.autograd.functional.jacobian(lambda u: eq.prim(u, gas), U0)  # [5 (W), 5 (U)]

    def f1(Ux):
        G = torch.zeros(3, 5, dtype=torch.float64)
        G = G.index_copy(0, torch.tensor([0]), (dWdU @ Ux).unsqueeze(0))
        return eq.flux_visc(eq.prim(U0, gas), G, gas)[0]  # flux in direction x1

    B = torch.autograd.functional.jacobian(f1, torch.zeros(5, dtype=torch.float64))
    lam = np.linalg.eigvals(B.numpy())
    assert np.abs(lam.imag).max() < 1e-12
    lam_max = lam.real.max()
    assert abs(lam_max - ratio * gas.mu / float(U0[0])) < 1e-12 * lam_max
