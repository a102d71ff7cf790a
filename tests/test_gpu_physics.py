"""Properties of the CUDA path at full configuration sizes, where the oracle is
too slow to follow: free-stream preservation on the curved C4 mesh (24^3,
N = 7, 50 steps), the order of accuracy on the C4 manufactured solution,
discrete conservation over many steps, and the kinetic-energy rate."""
import math

import numpy as np
import pytest
import torch

import workloads as wl

from test_gpu_parity import DEV, _solver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
def test_c4a_freestream_full_size(precision, tol):
    """C4a: [-1,1]^3, 24^3 curved elements, N = Ngeo = 7, free stream, 50 steps."""
    N = 7
    mesh = wl.box_mesh((24, 24, 24), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3)
    s = _solver(dict(N=N, Ngeo=N, riemann=1, bc_exact=1, precision=precision), mesh)
    U0 = torch.tensor(wl.freestream(mesh.node_coords(N, 0)), device=DEV, dtype=s.dtype)
    U = U0.clone()
    dt = 0.5 * s.reduce(U)["dt_max"]
    s.run(U, 50, dt)
    err = float((U - U0).abs().max() / U0.abs().max())
    s.close()
    assert err < tol, err


def _mms_error(N, nel, t_end):
    mesh = wl.box_mesh((nel,) * 3, lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3)
    s = _solver(dict(N=N, Ngeo=N, riemann=1, bc_exact=2, source=True), mesh)
    x = mesh.node_coords(N, 0)
    U = torch.tensor(wl.manufactured(x, 0.0), device=DEV)
    dt0 = 0.5 * s.reduce(U)["dt_max"]
    nsteps = int(math.ceil(t_end / dt0))
    s.run(U, nsteps, t_end / nsteps)
    Ue = torch.tensor(wl.manufactured(x, t_end), device=DEV)
    s.close()
    return float(((U[:, 0] - Ue[:, 0]) ** 2).mean().sqrt())


@pytest.mark.parametrize("N", [2, 3, 4])
def test_c4b_manufactured_order(N):
    """C4b on the curved mesh with Dirichlet data and the source term: the nodal
    RMS error of rho after t = 0.2 converges at order ~N+1 (finest pair >= N+0.5)."""
    errs = [_mms_error(N, nel, 0.2) for nel in (6, 12, 24)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[0] > errs[1] > errs[2]
    assert orders[-1] > N + 0.5, (errs, orders)


def test_conservation_and_ke_rate_long_run():
    """Periodic TGV, 8^3, N = 5: mass, momentum and energy conserved to round-off
    over 200 steps; dKE/dt from the reduction matches the KE history."""
    N = 5
    mesh = wl.box_mesh((8, 8, 8), Ngeo=1, reorient_seed=3)
    s = _solver(dict(N=N, riemann=1, mu=1 / 400.0), mesh)
    U = torch.tensor(wl.taylor_green(mesh.node_coords(N, 0)), device=DEV)
    r0 = s.reduce(U)
    dt = r0["dt_max"]
    kes, rates = [], []
    dU = torch.zeros_like(U)
    for k in range(201):
        if k % 50 == 0:
            r = s.reduce(U, s.rhs(U, k * dt))
            kes.append(r["kinetic_energy"])
            rates.append(r["dkedt"])
        if k < 200:
            s.step(U, dU, k * dt, dt)
    r1 = s.reduce(U)
    for key in ("mass", "mom_x", "mom_y", "mom_z", "energy"):
        assert abs(r1[key] - r0[key]) < 1e-12 * abs(r0["energy"]), key
    assert all(kes[i + 1] < kes[i] for i in range(len(kes) - 1))
    # the instantaneous rate is consistent with the KE drop over 50 steps (trapezoid, 1%)
    for i in range(len(kes) - 1):
        fd = (kes[i + 1] - kes[i]) / (50 * dt)
        assert abs(fd - 0.5 * (rates[i] + rates[i + 1])) < 0.01 * abs(fd), (fd, rates[i], rates[i + 1])
    s.close()
