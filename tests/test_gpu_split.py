"""Split-form DG on the GPU (Sec. 3.3, Eq. semiDiscreteSplit; Pirozzoli's
kinetic-energy-preserving two-point flux, Gauss-Lobatto nodes) through the C ABI
against the oracle's split form.

Right-hand sides use the rounding-sensitivity tolerance of test_gpu_parity (FP64;
1-ulp noise on the state and on the mesh coordinates) and its FP32 scaling of
test_gpu_precision; states after time steps 1e-12
relative L2 per conserved variable (FP64).  At the full 16^3, N = 7 size the
right-hand side is compared with the oracle in full, and the run is checked for
conservation and for the free stream on a curved mesh.
"""
import numpy as np
import pytest
import torch

import workloads as wl

from test_gpu_parity import DEV, _oracle, _solver, _state, per_var_rel, rhs_parity_ok, rounding_sensitivity

pytestmark = pytest.mark.gpu

KEP = 1
ECS = 2

CASES = [
    ("tgv_N1_roe", dict(nelem=(3, 3, 3), reorient_seed=1), dict(N=1, riemann=0), "tgv"),
    ("pert_N2_rusanov", dict(nelem=(3, 2, 3), reorient_seed=2), dict(N=2, riemann=3), "perturbed"),
    ("tgv_N3_roe", dict(nelem=(3, 3, 3), reorient_seed=3), dict(N=3, riemann=0), "tgv"),
    ("pert_N4_hllc", dict(nelem=(2, 3, 2), reorient_seed=4), dict(N=4, riemann=1), "perturbed"),
    ("pert_N5_roesmooth", dict(nelem=(2, 2, 3), reorient_seed=5), dict(N=5, riemann=2, mu=1 / 400.0), "perturbed"),
    ("pert_N6_hllc", dict(nelem=(2, 2, 2), reorient_seed=6), dict(N=6, riemann=1), "perturbed"),
    ("tgv_N7_hllc", dict(nelem=(2, 2, 3), reorient_seed=7), dict(N=7, riemann=1), "tgv"),
    ("curved_mms_N3", dict(nelem=(2, 3, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=3, mapping="sine",
                           periodic=(False, True, False), reorient_seed=8),
     dict(N=3, Ngeo=3, riemann=1, bc_exact=2, source=True), "manufactured"),
    ("curved_pert_N5", dict(nelem=(2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=5, mapping="sine",
                            periodic=(False,) * 3, reorient_seed=9),
     dict(N=5, Ngeo=5, riemann=0, bc_exact=1), "perturbed_small"),
]


def _kw(sk, precision=0):
    return dict(sk, node_type=1, split_form=KEP, precision=precision)


@pytest.mark.parametrize("name,mk,sk,state", CASES, ids=[c[0] for c in CASES])
def test_split_rhs_parity_fp64(name, mk, sk, state):
    mesh = wl.box_mesh(**mk)
    sk = _kw(sk)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = _state(state, mesh, sk["N"], 1)
    Ut = s.rhs(torch.tensor(U0, device=DEV), 0.1)
    ok, d, tol = rhs_parity_ok(Ut, dg, torch.tensor(U0), 0.1, mesh)
    s.close()
    assert ok, (d, tol)


@pytest.mark.parametrize("N,riem,nelem", [(7, 1, (3, 2, 2)), (4, 0, (3, 3, 2)), (2, 3, (3, 3, 3))])
def test_split_rhs_parity_fp32(N, riem, nelem):
    mesh = wl.box_mesh(nelem, reorient_seed=N)
    sk = _kw(dict(N=N, riemann=riem), precision=1)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = wl.perturbed(mesh.node_coords(N, 1), seed=3)
    Ut = s.rhs(torch.tensor(U0, device=DEV, dtype=torch.float32), 0.0)
    ref, parts = dg.rhs(torch.tensor(U0), 0.0, parts=True)
    scale = (ref.abs() + (parts["vol"] / dg.geo.J.unsqueeze(1)).abs()).transpose(0, 1).reshape(5, -1).norm(dim=1)
    sig = rounding_sensitivity(dg, torch.tensor(U0), 0.0, mesh=mesh) * 2.0 ** 29
    d = (Ut.double().cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    tol = torch.maximum(3e-6 * scale, 20 * sig)
    s.close()
    assert bool((d <= tol).all()), (d.tolist(), tol.tolist())


def test_split_differs_from_standard_on_gpu():
    """The split operator is a different discretisation: on the same LGL mesh the
    GPU split and standard right-hand sides must differ (a guard against the
    split flag being ignored)."""
    mesh = wl.box_mesh((2, 2, 2), reorient_seed=3)
    U0 = torch.tensor(wl.perturbed(mesh.node_coords(3, 1), seed=5), device=DEV)
    a = _solver(dict(N=3, node_type=1, riemann=1), mesh)
    b = _solver(_kw(dict(N=3, riemann=1)), mesh)
    ra, rb = a.rhs(U0), b.rhs(U0)
    a.close()
    b.close()
    assert (ra - rb).abs().max().item() > 1e-6 * ra.abs().max().item()


def test_split_rk_steps_match_oracle():
    """20 LSERK4(5) steps of the split form on the 4^3, N = 3 Taylor-Green case."""
    mesh = wl.box_mesh((4, 4, 4), Ngeo=1, reorient_seed=2)
    sk = _kw(dict(N=3, riemann=1))
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = wl.taylor_green(mesh.node_coords(3, 1))
    U = torch.tensor(U0, device=DEV)
    s.run(U, 20, 2e-3)
    Ur = dg.run(torch.tensor(U0), 20, 2e-3)
    err = per_var_rel(U, Ur)
    s.close()
    assert err < 1e-12, err


def test_split_freestream_curved_50_steps():
    N = 7
    mesh = wl.box_mesh((3, 3, 3), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3,
                       reorient_seed=4)
    s = _solver(_kw(dict(N=N, Ngeo=N, riemann=1, bc_exact=1)), mesh)
    U0 = torch.tensor(wl.freestream(mesh.node_coords(N, 1)), device=DEV)
    U = U0.clone()
    s.run(U, 50, 1e-3)
    err = (U - U0).abs().max().item()
    s.close()
    assert err < 1e-12, err


def test_split_full_size_rhs_and_invariants():
    """16^3, N = 7 LGL Taylor-Green (the timed size): the whole right-hand side
    against the oracle, then 50 steps conserving mass, momentum and energy with
    decaying kinetic energy."""
    N = 7
    mesh = wl.box_mesh((16, 16, 16), Ngeo=1)
    sk = _kw(dict(N=N, riemann=1))
    s = _solver(sk, mesh)
    U0 = wl.taylor_green(mesh.node_coords(N, 1))
    U = torch.tensor(U0, device=DEV)
    Ut = s.rhs(U, 0.0)
    dg = _oracle(sk, mesh)
    ok, d, tol = rhs_parity_ok(Ut, dg, torch.tensor(U0), 0.0, mesh)
    assert ok, (d, tol)
    del dg
    r0 = s.reduce(U)
    s.run(U, 50, r0["dt_max"])
    r1 = s.reduce(U)
    for key in ("mass", "mom_x", "mom_y", "mom_z", "energy"):
        assert abs(r1[key] - r0[key]) < 1e-12 * max(1.0, abs(r0["energy"])), key
    assert r1["kinetic_energy"] < r0["kinetic_energy"]
    s.close()


def test_split_unsupported_combinations():
    from paper_1910_02858_gb300 import flexi as F

    mesh = wl.box_mesh((2, 2, 2), Ngeo=1)
    for kw in (dict(N=3, node_type=0, split_form=KEP), dict(N=3, node_type=1, split_form=KEP, precision=2),
               dict(N=3, node_type=1, split_form=KEP, precision=3)):
        with pytest.raises(F.FlexiError) as ei:
            _solver(kw, mesh)
        assert ei.value.code == F.FLEXI_EUNSUPPORTED
    with pytest.raises(F.FlexiError) as ei:
        _solver(dict(N=3, node_type=1, split_form=3), mesh)
    assert ei.value.code == F.FLEXI_EINVAL
    with pytest.raises(F.FlexiError) as ei:
        _solver(dict(N=3, node_type=0, split_form=ECS), mesh)
    assert ei.value.code == F.FLEXI_EUNSUPPORTED
    with pytest.raises(F.FlexiError) as ei:
        _solver(dict(N=3, node_type=1, riemann=5), mesh)
    assert ei.value.code == F.FLEXI_EINVAL
    # the split-form adjoint runs (its parity with the oracle: test_gpu_adjoint_bc.py)
    s = _solver(dict(N=3, node_type=1, split_form=KEP, riemann=0, adjoint=True), mesh)
    U = torch.tensor(wl.taylor_green(mesh.node_coords(3, 1)), device=DEV)
    lam = torch.ones_like(U)
    out = torch.empty_like(U)
    F.flexi_rhs_adjoint(s.ctx, U, lam, out, 0.0, torch.cuda.current_stream())
    s.close()
    assert bool(torch.isfinite(out).all())



# ---------------------------------------------------------------------------
# entropy-conservative split form (Chandrashekar) and the EC surface flux
# ---------------------------------------------------------------------------
EC_CASES = [
    ("ec_tgv_N2_ecflux", dict(nelem=(3, 2, 3), reorient_seed=2), dict(N=2, riemann=4), "tgv"),
    ("ec_pert_N3_hllc", dict(nelem=(3, 3, 3), reorient_seed=3), dict(N=3, riemann=1), "perturbed"),
    ("ec_pert_N5_roe", dict(nelem=(2, 2, 3), reorient_seed=5), dict(N=5, riemann=0), "perturbed"),
    ("ec_tgv_N7_ecflux", dict(nelem=(2, 2, 3), reorient_seed=7), dict(N=7, riemann=4), "tgv"),
    ("ec_curved_N4_ecflux", dict(nelem=(2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=4, mapping="sine",
                                 periodic=(False,) * 3, reorient_seed=9),
     dict(N=4, Ngeo=4, riemann=4, bc_exact=1), "perturbed_small"),
]


@pytest.mark.parametrize("name,mk,sk,state", EC_CASES, ids=[c[0] for c in EC_CASES])
def test_ec_split_rhs_parity_fp64(name, mk, sk, state):
    mesh = wl.box_mesh(**mk)
    sk = dict(sk, node_type=1, split_form=ECS, precision=0)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = _state(state, mesh, sk["N"], 1)
    Ut = s.rhs(torch.tensor(U0, device=DEV), 0.1)
    ok, d, tol = rhs_parity_ok(Ut, dg, torch.tensor(U0), 0.1, mesh)
    s.close()
    assert ok, (d, tol)


def test_ec_split_rhs_parity_fp32():
    mesh = wl.box_mesh((3, 2, 2), reorient_seed=7)
    sk = dict(N=7, riemann=4, node_type=1, split_form=ECS, precision=1)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = wl.perturbed(mesh.node_coords(7, 1), seed=3)
    Ut = s.rhs(torch.tensor(U0, device=DEV, dtype=torch.float32), 0.0)
    ref, parts = dg.rhs(torch.tensor(U0), 0.0, parts=True)
    scale = (ref.abs() + (parts["vol"] / dg.geo.J.unsqueeze(1)).abs()).transpose(0, 1).reshape(5, -1).norm(dim=1)
    sig = rounding_sensitivity(dg, torch.tensor(U0), 0.0, mesh=mesh) * 2.0 ** 29
    d = (Ut.double().cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    tol = torch.maximum(3e-6 * scale, 20 * sig)
    s.close()
    assert bool((d <= tol).all()), (d.tolist(), tol.tolist())


def _entropy_rate(U, Ut, wJ, gamma=1.4):
    """sum_nodes wJ v . U_t with the entropy variables v of S = -rho s/(gamma - 1)."""
    rho = U[:, 0]
    u = U[:, 1:4] / rho.unsqueeze(1)
    p = (gamma - 1.0) * (U[:, 4] - 0.5 * rho * (u * u).sum(1))
    s = torch.log(p) - gamma * torch.log(rho)
    beta = rho / p
    v = torch.cat([((gamma - s) / (gamma - 1.0) - 0.5 * beta * (u * u).sum(1)).unsqueeze(1), beta.unsqueeze(1) * u,
                   -beta.unsqueeze(1)], 1)
    t = wJ.unsqueeze(1) * v * Ut
    return float(t.sum()), float(t.abs().sum())


@pytest.mark.parametrize("nelem,N,seed", [((4, 4, 4), 5, 1), ((16, 16, 16), 7, 2)])
def test_ec_split_conserves_entropy_on_gpu(nelem, N, seed):
    """Inviscid periodic flow with a rough state (random nodal values): the GPU's EC
    split form with the EC surface flux conserves the discrete entropy to round-off,
    also at the timed size (16^3, N = 7); with the HLLC surface flux entropy decays."""
    mesh = wl.box_mesh(nelem, reorient_seed=seed)
    x = mesh.node_coords(N, 1)
    rng = np.random.default_rng(seed)
    sh = x[:, 0].shape
    U0 = wl.prim_to_cons_np(1 + 0.2 * rng.random(sh), 0.3 * rng.normal(size=sh), 0.3 * rng.normal(size=sh),
                            0.3 * rng.normal(size=sh), 1 + 0.2 * rng.random(sh), 1.4)
    U = torch.tensor(U0, device=DEV)
    from oracle.basis import Basis  # quadrature weights of the entropy sum (Cartesian elements)
    b = Basis(N, 1)
    h = 2 * np.pi / nelem[0]
    w1 = torch.tensor(b.w_np, device=DEV)
    wJ = (w1.view(1, -1, 1, 1) * w1.view(1, 1, -1, 1) * w1.view(1, 1, 1, -1)) * (h / 2) ** 3
    res = {}
    for riem in (4, 1):
        s = _solver(dict(N=N, node_type=1, riemann=riem, split_form=ECS, mu=0.0), mesh)
        res[riem] = _entropy_rate(U, s.rhs(U), wJ)
        s.close()
    assert abs(res[4][0]) < 1e-11 * res[4][1], res
    assert res[1][0] < -1e-4 * res[1][1], res
