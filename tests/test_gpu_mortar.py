"""Mortar interfaces of non-conforming meshes on the GPU (Sec. "Non-conforming
meshes") through flexi_mesh_init_mortar, against the oracle's mortar treatment.

Right-hand sides use the rounding-sensitivity tolerance of test_gpu_parity (1-ulp
noise on the state and on the mesh coordinates, 20 sigma; FP32 scaled by 2^29);
states after time steps 1e-12 relative L2 per conserved variable (FP64)."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.dgsem import DGSEM, HLLC, ROE, RUSANOV, Params

from test_gpu_parity import DEV, per_var_rel, rounding_sensitivity

pytestmark = pytest.mark.gpu


def _solver(sk, mesh):
    from paper_1910_02858_gb300 import Solver, SolverConfig

    return Solver(SolverConfig(**sk), mesh.coords, mesh.conn, device=DEV, mortars=mesh.mortars)


def _oracle(sk, mesh):
    r = {0: ROE, 1: HLLC, 2: ROE, 3: RUSANOV}[sk.get("riemann", 0)]
    return DGSEM(Params(N=sk["N"], node_type=sk.get("node_type", 0), riemann=r, smooth_roe=sk.get("riemann", 0) == 2,
                        mu=sk.get("mu", 1 / 1600.0), bc_exact=sk.get("bc_exact", 0), source=sk.get("source", False),
                        split="pirozzoli" if sk.get("split_form", 0) == 1 else "",
                        lifting="br2" if sk.get("lifting", 0) == 1 else "br1", eta_br2=sk.get("eta_br2", 2.0)),
                 mesh.coords, mesh.conn, mesh.mortars)


def _sens(dg, U0, t, mesh, scale=1.0):
    sig_u = rounding_sensitivity(dg, U0, t)
    ref = dg.rhs(U0, t)
    rng = np.random.default_rng(4321)
    sig_x = torch.zeros(5, dtype=torch.float64)
    for _ in range(2):
        coords = mesh.coords * (1 + 2.2e-16 * (2 * rng.random(mesh.coords.shape) - 1))
        dgx = DGSEM(dg.p, coords, mesh.conn, mesh.mortars)
        sig_x = torch.maximum(sig_x, (dgx.rhs(U0, t) - ref).transpose(0, 1).reshape(5, -1).norm(dim=1))
    return torch.maximum(sig_u, sig_x) * scale


def _check_rhs(Ut, dg, U0, t, mesh, fp32=False):
    ref, parts = dg.rhs(U0, t, parts=True)
    scale = (ref.abs() + (parts["vol"] / dg.geo.J.unsqueeze(1)).abs()).transpose(0, 1).reshape(5, -1).norm(dim=1)
    sig = _sens(dg, U0, t, mesh, 2.0 ** 29 if fp32 else 1.0)
    d = (Ut.double().cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    tol = torch.maximum((3e-6 if fp32 else 1e-12) * scale, 20 * sig)
    return bool((d <= tol).all()), d.tolist(), tol.tolist()


CASES = [
    # (name, mesh kwargs, solver kwargs)
    ("t1_lg_N3_hllc", dict(refine=(1, 2, 1), ny=1, nz=2, reorient_seed=1), dict(N=3, riemann=1)),
    ("t2_lgl_N4_roe", dict(refine=(1, 1, 2), ny=2, nz=1, reorient_seed=2), dict(N=4, node_type=1, riemann=0)),
    ("t3_lg_N2_rusanov", dict(refine=(2, 2, 2), ny=1, nz=1, reorient_seed=3), dict(N=2, riemann=3)),
    ("t3_lg_N7_hllc", dict(refine=(1, 2, 2), ny=1, nz=1, reorient_seed=4), dict(N=7, riemann=1)),
    ("t3_lgl_N5_roesmooth", dict(refine=(1, 2, 2), ny=1, nz=1, reorient_seed=5),
     dict(N=5, node_type=1, riemann=2, mu=1 / 400.0)),
    ("t3_curved_lg_N4", dict(refine=(2, 2, 2), ny=1, nz=1, reorient_seed=6, mapping="sine", Ngeo=4),
     dict(N=4, Ngeo=4, riemann=1)),
    ("t1_curved_lgl_N6", dict(refine=(1, 2, 1), ny=1, nz=2, reorient_seed=7, mapping="sine", Ngeo=3),
     dict(N=6, Ngeo=3, node_type=1, riemann=1)),
    ("t3_split_lgl_N3", dict(refine=(2, 2, 2), ny=1, nz=1, reorient_seed=8), dict(N=3, node_type=1, riemann=1,
                                                                                 split_form=1)),
    ("t2_dirichlet_mms_N3", dict(refine=(1, 1, 2), ny=1, nz=2, reorient_seed=9, periodic=(False, True, True),
                                 mapping="sine", Ngeo=3),
     dict(N=3, Ngeo=3, riemann=1, bc_exact=2, source=True)),
]


def _state(mesh, N, nt, kind="perturbed"):
    x = mesh.node_coords(N, nt)
    if kind == "manufactured":
        return wl.manufactured(x, 0.0)
    return wl.perturbed(np.pi * x, seed=11)


@pytest.mark.parametrize("name,mk,sk", CASES, ids=[c[0] for c in CASES])
def test_mortar_rhs_parity_fp64(name, mk, sk):
    mesh = wl.mortar_box_mesh(**mk)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = _state(mesh, sk["N"], sk.get("node_type", 0), "manufactured" if sk.get("source") else "perturbed")
    Ut = s.rhs(torch.tensor(U0, device=DEV), 0.1)
    ok, d, tol = _check_rhs(Ut, dg, torch.tensor(U0), 0.1, mesh)
    s.close()
    assert ok, (d, tol)


@pytest.mark.parametrize("prec", [1, 2])
def test_mortar_rhs_parity_fp32(prec):
    mesh = wl.mortar_box_mesh(refine=(2, 2, 2), ny=1, nz=1, reorient_seed=3)
    sk = dict(N=5, riemann=1, precision=prec)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = _state(mesh, 5, 0)
    Ut = s.rhs(torch.tensor(U0, device=DEV, dtype=torch.float32), 0.0)
    ok, d, tol = _check_rhs(Ut, dg, torch.tensor(U0), 0.0, mesh, fp32=True)
    s.close()
    assert ok, (d, tol)


def test_mortar_rk_steps_match_oracle():
    mesh = wl.mortar_box_mesh(refine=(2, 2, 2), ny=2, nz=2, nx=1, reorient_seed=4, mapping="sine", Ngeo=3)
    sk = dict(N=3, Ngeo=3, riemann=1)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = _state(mesh, 3, 0)
    U = torch.tensor(U0, device=DEV)
    s.run(U, 20, 1e-3)
    Ur = dg.run(torch.tensor(U0), 20, 1e-3)
    err = per_var_rel(U, Ur)
    s.close()
    assert err < 1e-12, err


@pytest.mark.parametrize("nt", [0, 1])
def test_mortar_freestream_curved_50_steps(nt):
    N = 7
    mesh = wl.mortar_box_mesh(refine=(2, 2, 2), ny=1, nz=1, reorient_seed=5, mapping="sine", Ngeo=N)
    s = _solver(dict(N=N, Ngeo=N, node_type=nt, riemann=1), mesh)
    U0 = torch.tensor(wl.freestream(mesh.node_coords(N, nt)), device=DEV)
    U = U0.clone()
    s.run(U, 50, 1e-3)
    err = (U - U0).abs().max().item()
    s.close()
    assert err < 1e-12, err


def test_mortar_conservation_100_steps():
    """Periodic curved mesh with type-3 mortars at both interfaces, N = 7: mass,
    momentum and energy stay constant over 100 steps."""
    N = 7
    mesh = wl.mortar_box_mesh(refine=(2, 2, 2), ny=2, nz=2, nx=1, reorient_seed=6, mapping="sine", Ngeo=N)
    s = _solver(dict(N=N, Ngeo=N, riemann=1), mesh)
    U = torch.tensor(_state(mesh, N, 0), device=DEV)
    r0 = s.reduce(U)
    s.run(U, 100, 0.5 * r0["dt_max"])
    r1 = s.reduce(U)
    for key in ("mass", "mom_x", "mom_y", "mom_z", "energy"):
        assert abs(r1[key] - r0[key]) < 1e-12 * max(1.0, abs(r0["energy"])), key
    s.close()


def test_mortar_errors():
    from paper_1910_02858_gb300 import flexi as F

    mesh = wl.mortar_box_mesh(refine=(2, 2, 2), ny=1, nz=1)
    bad = wl.mortar_box_mesh(refine=(2, 2, 2), ny=1, nz=1)
    bad.mortars = bad.mortars.copy()
    bad.mortars[0, 5] = 8  # orientation code out of range
    with pytest.raises(F.FlexiError) as ei:
        _solver(dict(N=2), bad)
    assert ei.value.code == F.FLEXI_EMESH
    bad.mortars = mesh.mortars.copy()
    bad.mortars[0, 3], bad.mortars[1, 3] = mesh.mortars[1, 3], mesh.mortars[0, 3]  # rows disagree with conn
    with pytest.raises(F.FlexiError) as ei:
        _solver(dict(N=2), bad)
    assert ei.value.code == F.FLEXI_EMESH
    with pytest.raises(F.FlexiError) as ei:  # mortar sides but no mortar rows
        from paper_1910_02858_gb300 import Solver, SolverConfig

        Solver(SolverConfig(N=2), mesh.coords, mesh.conn, device=DEV)
    assert ei.value.code == F.FLEXI_EMESH
    s = _solver(dict(N=2, riemann=0, adjoint=True, precision=2), mesh)  # no reverse of the tensor-core sweeps
    U = torch.tensor(wl.freestream(mesh.node_coords(2, 0)), device=DEV, dtype=torch.float32)
    with pytest.raises(F.FlexiError) as ei:
        F.flexi_rhs_adjoint(s.ctx, U, torch.ones_like(U), torch.empty_like(U), 0.0, torch.cuda.current_stream())
    s.close()
    assert ei.value.code == F.FLEXI_EUNSUPPORTED


ADJ_CASES = [
    ("t1_lg_N3_roesmooth", dict(refine=(1, 2, 1), ny=1, nz=2, reorient_seed=1), dict(N=3, riemann=2, mu=1 / 400.0)),
    ("t3_lgl_N4_hllc", dict(refine=(1, 2, 2), ny=1, nz=1, reorient_seed=5),
     dict(N=4, node_type=1, riemann=1, mu=1 / 400.0)),
    ("t2_curved_lg_N2_rusanov", dict(refine=(1, 1, 2), ny=2, nz=1, reorient_seed=2, mapping="sine", Ngeo=2),
     dict(N=2, Ngeo=2, riemann=3, mu=1 / 400.0)),
    ("t3_split_lgl_N3", dict(refine=(2, 2, 2), ny=1, nz=1, reorient_seed=8),
     dict(N=3, node_type=1, riemann=1, split_form=1, mu=1 / 400.0)),
    ("t2_dirichlet_mms_N3", dict(refine=(1, 1, 2), ny=1, nz=2, reorient_seed=9, periodic=(False, True, True),
                                 mapping="sine", Ngeo=3),
     dict(N=3, Ngeo=3, riemann=2, bc_exact=2, source=True, mu=1 / 400.0)),
    ("t3_br2_lg_N3_hllc", dict(refine=(1, 2, 2), ny=1, nz=1, reorient_seed=3),
     dict(N=3, riemann=1, lifting=1, eta_br2=2.0, mu=1 / 400.0)),
    ("t1_br2_lgl_N4_eta5", dict(refine=(1, 2, 1), ny=1, nz=2, reorient_seed=6, mapping="sine", Ngeo=2),
     dict(N=4, Ngeo=2, node_type=1, riemann=2, lifting=1, eta_br2=5.0, mu=1 / 400.0)),
]


@pytest.mark.parametrize("name,mk,sk", ADJ_CASES, ids=[c[0] for c in ADJ_CASES])
def test_mortar_rhs_adjoint_vs_oracle(name, mk, sk):
    """Discrete adjoint on mortar meshes: the transposed interpolation of the big
    side's state and gradients and the transposed projections of its lifting and
    numerical fluxes, against the oracle's reverse-mode derivative."""
    mesh = wl.mortar_box_mesh(**mk)
    s = _solver(dict(sk, adjoint=True), mesh)
    dg = _oracle(sk, mesh)
    U0 = _state(mesh, sk["N"], sk.get("node_type", 0), "manufactured" if sk.get("source") else "perturbed")
    lam = np.random.default_rng(6).normal(size=U0.shape)
    out = s.rhs_adjoint(torch.tensor(U0, device=DEV), torch.tensor(lam, device=DEV), 0.1)
    ref = dg.rhs_vjp(torch.tensor(U0), 0.1, torch.tensor(lam))
    s.close()
    d = (out.cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    r = ref.transpose(0, 1).reshape(5, -1).norm(dim=1)
    assert float((d / r).max()) < 1e-10, (d / r).tolist()


@pytest.mark.parametrize("ci", [0, 2])
def test_mortar_adjoint_dot_product(ci):
    """Central-difference dot-product test on a mortar mesh (no oracle)."""
    name, mk, sk = ADJ_CASES[ci]
    mesh = wl.mortar_box_mesh(**mk)
    s = _solver(dict(sk, adjoint=True), mesh)
    U0 = torch.tensor(_state(mesh, sk["N"], sk.get("node_type", 0)), device=DEV)
    g = torch.Generator(device="cpu").manual_seed(8)
    v = torch.randn(U0.shape, generator=g, dtype=torch.float64).to(DEV)
    lam = torch.randn(U0.shape, generator=g, dtype=torch.float64).to(DEV)
    eps = 1e-6
    Jv = (s.rhs(U0 + eps * v, 0.1) - s.rhs(U0 - eps * v, 0.1)) / (2 * eps)
    a = float((lam * Jv).sum())
    b = float((s.rhs_adjoint(U0, lam, 0.1) * v).sum())
    s.close()
    assert abs(a - b) < 1e-6 * abs(b), (a, b)
