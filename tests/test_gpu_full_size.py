"""Full-size workloads on the CUDA path, checked through properties that hold at any
size (the oracle needs minutes per right-hand side at these sizes).

- Curved mesh (24^3 elements mapped by x_i = xi_i + 0.1 prod_j sin(pi xi_j), N = Ngeo = 7,
  curl-form metrics, Dirichlet sides, 7,077,888 DOF): the free stream is preserved over
  50 LSERK4(5) steps (Sec. 3.1: the curl form makes the metric identities hold
  discretely); the right-hand side of the manufactured solution, sampled exactly at the
  nodes at time t with its source term and exact-state boundaries, reproduces the exact
  dU/dt to the truncation error of an N = 7 discretisation on this mesh.
- Taylor-Green 32^3, N = 5 Gauss (7,077,888 DOF), FP64: discrete conservation of the
  right-hand side, sum over nodes of w_i w_j w_k J U_t = 0 for mass, momentum and energy
  (the quadrature weights and the Cartesian J = (h/2)^3 written out here), and of the
  conserved totals over ten steps.  The face fluxes cancel between neighbours in exact
  arithmetic; the round-off left is relative to the fluxes themselves, so each variable's
  sum is measured against (2/h) sum wJ sum_d |F^c_d| (the magnitude of its convective
  fluxes), not against the small low-Mach U_t.
"""
import math

import numpy as np
import pytest
import torch

import workloads as wl

from test_gpu_parity import DEV, _solver

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def curved_mesh():
    return wl.box_mesh((24, 24, 24), lo=(-1.0,) * 3, hi=(1.0,) * 3, Ngeo=7, mapping="sine", periodic=(False,) * 3)


def test_c4_freestream_preserved_full_size(curved_mesh):
    N = 7
    s = _solver(dict(N=N, Ngeo=N, riemann=1, bc_exact=1), curved_mesh)
    U0 = torch.tensor(wl.freestream(curved_mesh.node_coords(N, 0)), device=DEV)
    U = U0.clone()
    dt = s.reduce(U)["dt_max"]
    s.run(U, 50, dt)
    torch.cuda.synchronize()
    dev = ((U - U0).abs().amax(dim=(0, 2, 3, 4)) / U0.abs().amax(dim=(0, 2, 3, 4))).max().item()
    s.close()
    print("C4 free stream, 50 steps: largest relative deviation %.2e" % dev)
    assert dev < 1e-11, dev


def test_c4_manufactured_consistency_full_size(curved_mesh):
    N, t = 7, 0.3
    s = _solver(dict(N=N, Ngeo=N, riemann=1, bc_exact=2, source=True), curved_mesh)
    x = curved_mesh.node_coords(N, 0)
    U = torch.tensor(wl.manufactured(x, t), device=DEV)
    Ut = s.rhs(U, t).cpu()
    s.close()
    # exact dU/dt of rho = 2 + 0.1 sin(pi (x + y + z - 2t)), m = (rho, rho, rho), rho E = rho^2
    phase = math.pi * (x[:, 0] + x[:, 1] + x[:, 2] - 2.0 * t)  # node_coords: [K, 3, k, j, i]
    rho = 2.0 + 0.1 * np.sin(phase)
    rho_t = -0.2 * math.pi * np.cos(phase)
    exact = np.stack([rho_t, rho_t, rho_t, rho_t, 2.0 * rho * rho_t], axis=1)
    exact = torch.tensor(exact)
    d = (Ut - exact).transpose(0, 1).reshape(5, -1).norm(dim=1)
    r = exact.transpose(0, 1).reshape(5, -1).norm(dim=1)
    err = (d / r).max().item()
    print("C4 manufactured solution: relative L2 of U_t - dU/dt %.2e" % err)
    assert err < 1e-6, (d / r).tolist()


def test_c3_conservation_full_size():
    N = 5
    mesh = wl.box_mesh((32, 32, 32), Ngeo=1)
    s = _solver(dict(N=N, riemann=1), mesh)
    U = torch.tensor(wl.taylor_green(mesh.node_coords(N, 0)), device=DEV)
    Ut = s.rhs(U, 0.0)
    w = np.polynomial.legendre.leggauss(N + 1)[1]
    h = 2.0 * math.pi / 32
    wJ = torch.tensor(np.einsum("k,j,i->kji", w, w, w) * (h / 2) ** 3, device=DEV)
    tot = (wJ * Ut).sum(dim=(0, 2, 3, 4))
    # magnitude of the convective fluxes per variable: |m_d|, |m_c u_d + p delta_cd|, |u_d (E + p)|
    rho, m, E = U[:, 0], U[:, 1:4], U[:, 4]
    u = m / rho.unsqueeze(1)
    p = 0.4 * (E - 0.5 * (m * u).sum(1))
    fmag = torch.stack([m.abs().sum(1)] +
                       [sum((m[:, c] * u[:, d] + (p if c == d else 0.0)).abs() for d in range(3)) for c in range(3)] +
                       [(u * (E + p).unsqueeze(1)).abs().sum(1)], dim=1)
    scale = (2.0 / h) * (wJ * fmag).sum(dim=(0, 2, 3, 4))
    rel = (tot.abs() / scale).max().item()
    print("C3 sum wJ U_t relative to the convective flux magnitude %.2e" % rel, (tot / scale).tolist())
    assert rel < 1e-13, (tot / scale).tolist()
    r0 = s.reduce(U)
    s.run(U, 10, 0.5 * r0["dt_max"])
    r1 = s.reduce(U)
    s.close()
    for key in ("mass", "mom_x", "mom_y", "mom_z", "energy"):
        assert abs(r1[key] - r0[key]) < 1e-12 * max(1.0, abs(r0["energy"])), key
