"""FP32 precision forms of the CUDA path: FP32 storage and flux arithmetic with
the D_hat line sweeps on the FP32 pipes, on tensor cores in TF32 (3-pass
split) or in BF16 (3-term split), all accumulating in FP32.

Right-hand sides are compared with the FP64 oracle using the tolerance of
test_gpu_parity scaled to FP32 rounding (unit roundoff 2^-24 instead of
2^-53, a factor 2^29), and states after 100 steps of the C3 workload
(Taylor-Green, 32^3, N = 5) against the FP64 CUDA path, with the 1e-5
relative L2 budget per conserved variable (momentum components measured
against the norm of the momentum vector, since the Taylor-Green w-momentum
starts at zero).
"""
import numpy as np
import pytest
import torch

import workloads as wl

from test_gpu_parity import DEV, _oracle, _solver, rounding_sensitivity

pytestmark = pytest.mark.gpu

FORMS = {"fp32": 1, "tf32x3": 2, "bf16x3": 3}


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("N,nt,riem,nelem", [(7, 0, 1, (3, 2, 2)), (5, 0, 0, (2, 3, 3)), (3, 1, 1, (3, 3, 3)),
                                              (2, 0, 2, (3, 2, 3)), (1, 0, 1, (3, 3, 3))])
def test_rhs_fp32_forms_vs_oracle(form, N, nt, riem, nelem):
    mesh = wl.box_mesh(nelem, reorient_seed=N)
    sk = dict(N=N, node_type=nt, riemann=riem, precision=FORMS[form])
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = wl.perturbed(mesh.node_coords(N, nt), seed=3)
    Ut = s.rhs(torch.tensor(U0, device=DEV, dtype=torch.float32), 0.0)
    ref, parts = dg.rhs(torch.tensor(U0), 0.0, parts=True)
    scale = (ref.abs() + (parts["vol"] / dg.geo.J.unsqueeze(1)).abs()).transpose(0, 1).reshape(5, -1).norm(dim=1)
    sig = rounding_sensitivity(dg, torch.tensor(U0), 0.0, mesh=mesh) * 2.0 ** 29
    d = (Ut.double().cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    tol = torch.maximum(3e-6 * scale, 20 * sig)
    s.close()
    assert bool((d <= tol).all()), (d.tolist(), tol.tolist())


def test_c3_fp32_forms_100_steps_vs_fp64():
    """C3: TGV 32^3, N = 5, HLLC, 100 steps; every FP32 form within 1e-5 relative
    L2 per conserved variable of the FP64 path, kinetic energy within 1e-5, and the
    kinetic-energy dissipation rate dKE/dt within 2e-3.  The rate sum_nodes wJ dKE/dU . U_t
    is 0.116 while its terms carry the large constant pressure p0 = 71 (low Mach):
    measured agreement 2e-5 (FP32) to 6e-4 (BF16x3), so 2e-3 leaves a factor 3."""
    N = 5
    mesh = wl.box_mesh((32, 32, 32), Ngeo=1)
    U0 = wl.taylor_green(mesh.node_coords(N, 0))
    s64 = _solver(dict(N=N, riemann=1, precision=0), mesh)
    U64 = torch.tensor(U0, device=DEV)
    dt = s64.reduce(U64)["dt_max"]
    s64.run(U64, 100, dt)
    ke64 = s64.reduce(U64)["kinetic_energy"]
    rate64 = s64.reduce(U64, s64.rhs(U64))["dkedt"]
    s64.close()
    errs = {}
    for form, prec in FORMS.items():
        s = _solver(dict(N=N, riemann=1, precision=prec), mesh)
        U = torch.tensor(U0, device=DEV, dtype=torch.float32)
        s.run(U, 100, dt)
        d = (U.double() - U64).transpose(0, 1).reshape(5, -1).norm(dim=1)
        r = U64.transpose(0, 1).reshape(5, -1).norm(dim=1)
        r[1:4] = r[1:4].norm()  # momentum components against the momentum vector (w starts at 0)
        errs[form] = (d / r).tolist()
        ke = s.reduce(U)["kinetic_energy"]
        errs[form + "_ke"] = abs(ke - ke64) / ke64
        errs[form + "_rate"] = abs(s.reduce(U, s.rhs(U))["dkedt"] - rate64) / abs(rate64)
        s.close()
    for form in FORMS:
        assert max(errs[form]) < 1e-5, errs
        assert errs[form + "_ke"] < 1e-5, errs
        assert errs[form + "_rate"] < 2e-3, errs


@pytest.mark.parametrize("N", [3, 7])
def test_rhs_fp32_manufactured_source_curved(N):
    """C4b shape in the FP32 form: curved mesh, exact-state (Dirichlet) sides and the
    manufactured solution's source term (evaluated in FP32 after an FP64 phase
    reduction), at a time where the phase is not small; FP32 tolerance as above."""
    mesh = wl.box_mesh((2, 3, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3,
                       reorient_seed=N)
    sk = dict(N=N, Ngeo=N, riemann=1, bc_exact=2, source=True, precision=1)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    t = 0.37
    U0 = wl.manufactured(mesh.node_coords(N, 0), t)
    Ut = s.rhs(torch.tensor(U0, device=DEV, dtype=torch.float32), t)
    ref, parts = dg.rhs(torch.tensor(U0), t, parts=True)
    scale = (ref.abs() + (parts["vol"] / dg.geo.J.unsqueeze(1)).abs()).transpose(0, 1).reshape(5, -1).norm(dim=1)
    sig = rounding_sensitivity(dg, torch.tensor(U0), t, mesh=mesh) * 2.0 ** 29
    d = (Ut.double().cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    tol = torch.maximum(3e-6 * scale, 20 * sig)
    s.close()
    assert bool((d <= tol).all()), (d.tolist(), tol.tolist())
