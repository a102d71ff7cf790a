"""Discrete adjoint of the CUDA path (flexi_rhs_adjoint, flexi_adjoint_step and
the checkpointed torch.autograd.Function) against the oracle's reverse-mode
derivative, a forward-mode dot-product test and central finite differences."""
import math

import numpy as np
import pytest
import torch

import workloads as wl

from test_gpu_parity import DEV, _oracle, _solver

pytestmark = pytest.mark.gpu


def _state(mesh, N, seed=2):
    x = mesh.node_coords(N, 0)
    return wl.taylor_green(x) + 0.01 * (wl.perturbed(x, seed=seed) - wl.perturbed(x, seed=seed).mean())


@pytest.mark.parametrize("N,riem,nelem", [(2, 2, (2, 3, 2)), (3, 0, (3, 2, 2)), (5, 2, (2, 2, 2)), (7, 2, (2, 2, 1)),
                                          (1, 2, (3, 3, 3))])
def test_rhs_adjoint_vs_oracle(N, riem, nelem):
    mesh = wl.box_mesh(nelem, reorient_seed=N + 1)
    sk = dict(N=N, riemann=riem, mu=1 / 400.0, adjoint=True)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = _state(mesh, N)
    lam = np.random.default_rng(N).normal(size=U0.shape)
    out = s.rhs_adjoint(torch.tensor(U0, device=DEV), torch.tensor(lam, device=DEV))
    ref = dg.rhs_vjp(torch.tensor(U0), 0.0, torch.tensor(lam))
    d = (out.cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    r = ref.transpose(0, 1).reshape(5, -1).norm(dim=1)
    s.close()
    assert float((d / r).max()) < 1e-10, (d / r).tolist()


def test_adjoint_step_vs_oracle():
    N = 3
    mesh = wl.box_mesh((3, 2, 2), reorient_seed=4)
    sk = dict(N=N, riemann=2, mu=1 / 400.0, adjoint=True)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = _state(mesh, N)
    rng = np.random.default_rng(9)
    lamU0, lamdU0 = rng.normal(size=U0.shape), rng.normal(size=U0.shape)
    U = torch.tensor(U0, device=DEV)
    stages = torch.empty((5,) + U.shape, dtype=U.dtype, device=DEV)
    s.step_stages(U, torch.zeros_like(U), 0.0, 1e-3, stages)
    lamU, lamdU = torch.tensor(lamU0, device=DEV), torch.tensor(lamdU0, device=DEV)
    s.adjoint_step(stages, lamU, lamdU, 0.0, 1e-3)
    st_ref = []
    dg.rk_step(torch.tensor(U0), torch.zeros_like(torch.tensor(U0)), 0.0, 1e-3, stages_out=st_ref)
    rU, rdU = dg.adjoint_step(st_ref, torch.tensor(lamU0), torch.tensor(lamdU0), 0.0, 1e-3)
    assert float((lamU.cpu() - rU).norm() / rU.norm()) < 1e-12
    # the last reverse stage multiplies lam_dU by A_1 = 0: both sides are exactly zero
    assert float(lamdU.abs().max()) == 0.0 and float(rdU.abs().max()) == 0.0
    s.close()


def test_dot_product_with_finite_difference_jvp():
    """<lam, J v> from a central difference of flexi_rhs equals <J^T lam, v>."""
    N = 4
    mesh = wl.box_mesh((2, 2, 3), reorient_seed=2)
    s = _solver(dict(N=N, riemann=2, mu=1 / 400.0, adjoint=True), mesh)
    U0 = torch.tensor(_state(mesh, N), device=DEV)
    g = torch.Generator(device="cpu").manual_seed(5)
    v = torch.randn(U0.shape, generator=g, dtype=torch.float64).to(DEV)
    lam = torch.randn(U0.shape, generator=g, dtype=torch.float64).to(DEV)
    eps = 1e-6
    Jv = (s.rhs(U0 + eps * v) - s.rhs(U0 - eps * v)) / (2 * eps)
    a = float((lam * Jv).sum())
    b = float((s.rhs_adjoint(U0, lam) * v).sum())
    s.close()
    assert abs(a - b) < 1e-6 * abs(b), (a, b)


@pytest.fixture(scope="module")
def c5():
    """C5: TGV Re = 400, 8^3 periodic, N = 5 Gauss, Roe with smoothed |lambda|,
    40 steps x 5 stages at dt = 1e-3, checkpoints every 20 steps."""
    N = 5
    mesh = wl.box_mesh((8, 8, 8), Ngeo=1)
    sk = dict(N=N, riemann=2, mu=1 / 400.0, adjoint=True)
    s = _solver(sk, mesh)
    U0 = wl.taylor_green(mesh.node_coords(N, 0))
    yield mesh, s, sk, U0
    s.close()


def _ke(s, U):
    return s.reduce(U)["kinetic_energy"]


def _ke_nodes(U):
    return 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2) / U[:, 0]


def test_c5_gradient_fd_and_oracle(c5):
    from paper_1910_02858_gb300.adjoint import final_state

    mesh, s, sk, U0 = c5
    nsteps, dt = 40, 1e-3
    U0d = torch.tensor(U0, device=DEV, requires_grad=True)
    UT = final_state(U0d, s, nsteps, dt, 0.0, 20)
    # J = sum w J |m|^2 / (2 rho): its gradient with respect to U_T by the same reduction
    wJ = torch.tensor(_oracle(sk, mesh).quad_weights().numpy(), device=DEV).unsqueeze(1)
    J = (wJ[:, 0] * 0.5 * (UT[:, 1] ** 2 + UT[:, 2] ** 2 + UT[:, 3] ** 2) / UT[:, 0]).sum()
    Jv = J.detach().item()
    assert abs(Jv - _ke(s, UT.detach())) < 1e-12 * Jv
    J.backward()
    grad = U0d.grad.detach()
    # central finite differences (eps = 1e-6) in 16 seeded directions with unit
    # RMS per entry, so eps is the size of the perturbation of every DOF (with
    # unit-L2 directions over 553k entries the per-entry step would be 1.3e-9,
    # below the FP64 rounding floor of the 40-step evolution).  J(U+) - J(U-) is
    # summed term by term (subtracting two O(30) totals would leave the summation
    # rounding of each divided by 2 eps).
    errs = []
    for v in wl.random_directions(U0.shape, 16, seed0=1910, norm="rms"):
        vd = torch.tensor(v, device=DEV)
        Up = torch.tensor(U0, device=DEV) + 1e-6 * vd
        Um = torch.tensor(U0, device=DEV) - 1e-6 * vd
        s.run(Up, nsteps, dt)
        s.run(Um, nsteps, dt)
        fd = float((wJ[:, 0] * (_ke_nodes(Up) - _ke_nodes(Um))).sum()) / 2e-6
        ad = float((grad * vd).sum())
        errs.append(abs(fd - ad) / abs(ad))
    assert max(errs) < 1e-6, errs


def test_c5_gradient_vs_oracle_adjoint(c5):
    """Same workload, 4 steps with checkpoints every 2 steps, against the FP64 CPU
    adjoint of the oracle (reverse mode of the same discrete operator); the full
    40-step oracle gradient takes minutes on the host, so it is not repeated here."""
    from paper_1910_02858_gb300.adjoint import final_state

    mesh, s, sk, U0 = c5
    nsteps, dt = 4, 1e-3
    dg = _oracle(sk, mesh)
    wJ = torch.tensor(dg.quad_weights().numpy(), device=DEV)
    U0d = torch.tensor(U0, device=DEV, requires_grad=True)
    UT = final_state(U0d, s, nsteps, dt, 0.0, 2)
    J = (wJ * 0.5 * (UT[:, 1] ** 2 + UT[:, 2] ** 2 + UT[:, 3] ** 2) / UT[:, 0]).sum()
    J.backward()
    Jo, go = dg.gradient_ke(torch.tensor(U0), nsteps, dt)
    assert abs(Jo - J.detach().item()) < 1e-12 * abs(Jo)
    assert float((U0d.grad.cpu() - go).norm() / go.norm()) < 1e-10


def _c5_run(s, mesh, sk, U0, dtype):
    from paper_1910_02858_gb300.adjoint import final_state

    wJ = torch.tensor(_oracle(sk, mesh).quad_weights().numpy(), device=DEV, dtype=dtype)
    U0d = torch.tensor(U0, device=DEV, dtype=dtype, requires_grad=True)
    UT = final_state(U0d, s, 40, 1e-3, 0.0, 20)
    J = (wJ * 0.5 * (UT[:, 1] ** 2 + UT[:, 2] ** 2 + UT[:, 3] ** 2) / UT[:, 0]).sum()
    J.backward()
    return UT.detach().double().cpu(), U0d.grad.detach().double().cpu(), J.detach().item()


def test_c5_fp32_forward_and_adjoint_error(c5):
    """C5 in the FP32 form (forward and discrete adjoint in FP32 arithmetic)
    against the FP64 path: the final state (momentum components against the norm
    of the momentum vector), the functional and the gradient dJ/dU0 stay within
    the 1e-5 relative L2 budget of the precision form."""
    mesh, s64, sk, U0 = c5
    s32 = _solver(dict(sk, precision=1), mesh)
    U64, g64, J64 = _c5_run(s64, mesh, sk, U0, torch.float64)
    U32, g32, J32 = _c5_run(s32, mesh, sk, U0, torch.float32)
    s32.close()
    d = (U32 - U64).transpose(0, 1).reshape(5, -1).norm(dim=1)
    r = U64.transpose(0, 1).reshape(5, -1).norm(dim=1)
    r[1:4] = U64[:, 1:4].norm()
    assert float((d / r).max()) < 1e-5, (d / r).tolist()
    assert abs(J32 - J64) < 1e-5 * abs(J64)
    assert float((g32 - g64).norm() / g64.norm()) < 1e-5


def test_adjoint_needs_its_scratch():
    """Without flexi_params.adjoint the context holds no adjoint scratch and the
    adjoint calls report FLEXI_EUNSUPPORTED; with it they run."""
    from paper_1910_02858_gb300 import flexi as F

    mesh = wl.box_mesh((2, 2, 2))
    U = torch.tensor(_state(mesh, 2), device=DEV)
    lam = torch.ones_like(U)
    s = _solver(dict(N=2, riemann=2, mu=1 / 400.0), mesh)
    plain = s.query(F.Q_DEVICE_BYTES)
    with pytest.raises(F.FlexiError) as ei:
        s.rhs_adjoint(U, lam)
    s.close()
    assert ei.value.code == F.FLEXI_EUNSUPPORTED
    s = _solver(dict(N=2, riemann=2, mu=1 / 400.0, adjoint=True), mesh)
    assert s.query(F.Q_DEVICE_BYTES) > plain
    assert torch.isfinite(s.rhs_adjoint(U, lam)).all()
    s.close()
