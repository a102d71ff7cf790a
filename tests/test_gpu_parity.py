"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances.  States after time steps: 1e-12 relative L2 per conserved
variable (the bar for the FP64 path).  Right-hand sides: the operator output
is a difference of large terms (|vol/J| reaches 3e4 where U_t is 1e-3 for the
low-Mach Taylor-Green state), so two correct FP64 evaluations that round
differently disagree by the operator's own rounding sensitivity.  The test
measures that sensitivity sigma_v on the oracle itself: the larger change of U_t
under random 1-ulp relative perturbations of U, and under random 1-ulp relative
perturbations of the mesh node coordinates (both implementations compute the
metric terms from the coordinates with their own rounding; with the large
constant pressure of the low-Mach state multiplied by l_hat(+-1) ~ N(N+1)/2 on
Gauss-Lobatto faces, metric rounding dominates), and accepts, per variable,
||dU_t|| <= max(1e-12 ||(|U_t| + |vol/J|)||, 20 sigma_v).
"""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import equations as eq
from oracle.dgsem import DGSEM, EC, HLLC, ROE, RUSANOV, Params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_02858_gb300 import build as b

    b.build()
    from paper_1910_02858_gb300 import flexi as F

    F.lib()


def _solver(cfg_kw, mesh):
    from paper_1910_02858_gb300 import Solver, SolverConfig

    return Solver(SolverConfig(**cfg_kw), mesh.coords, mesh.conn, device=DEV)


def _oracle(cfg_kw, mesh):
    r = {0: ROE, 1: HLLC, 2: ROE, 3: RUSANOV, 4: EC}[cfg_kw.get("riemann", 0)]
    bc = cfg_kw.get("bc_exact", 0)
    return DGSEM(Params(N=cfg_kw["N"], node_type=cfg_kw.get("node_type", 0), riemann=r,
                        smooth_roe=cfg_kw.get("riemann", 0) == 2, mu=cfg_kw.get("mu", 1 / 1600.0),
                        Ma=cfg_kw.get("Ma", 0.1), bc_exact=bc, source=cfg_kw.get("source", False),
                        gamma=cfg_kw.get("gamma", 1.4), Pr=cfg_kw.get("Pr", 0.72),
                        split={0: "", 1: "pirozzoli", 2: "chandrashekar"}[cfg_kw.get("split_form", 0)],
                        lifting="br2" if cfg_kw.get("lifting", 0) == 1 else "br1", eta_br2=cfg_kw.get("eta_br2", 2.0)),
                 mesh.coords, mesh.conn)


def rounding_sensitivity(dg, U0, t, trials=2, mesh=None):
    """Per-variable L2 change of the oracle's U_t under 1-ulp relative noise on U
    and, given the mesh, on its node coordinates (the larger of the two)."""
    ref = dg.rhs(U0, t)
    g = torch.Generator().manual_seed(1234)
    sig = torch.zeros(5, dtype=torch.float64)
    for _ in range(trials):
        Up = U0 * (1 + 2.2e-16 * (2 * torch.rand(U0.shape, generator=g, dtype=torch.float64) - 1))
        sig = torch.maximum(sig, (dg.rhs(Up, t) - ref).transpose(0, 1).reshape(5, -1).norm(dim=1))
    if mesh is not None:
        rng = np.random.default_rng(4321)
        for _ in range(trials):
            coords = mesh.coords * (1 + 2.2e-16 * (2 * rng.random(mesh.coords.shape) - 1))
            dgx = DGSEM(dg.p, coords, mesh.conn)
            sig = torch.maximum(sig, (dgx.rhs(U0, t) - ref).transpose(0, 1).reshape(5, -1).norm(dim=1))
            del dgx
    return sig


def rhs_parity_ok(Ut_gpu, dg, U0, t, mesh=None):
    """Apply the right-hand-side tolerance described in the module docstring."""
    ref, parts = dg.rhs(U0, t, parts=True)
    scale = (ref.abs() + (parts["vol"] / dg.geo.J.unsqueeze(1)).abs()).transpose(0, 1).reshape(5, -1).norm(dim=1)
    sig = rounding_sensitivity(dg, U0, t, mesh=mesh)
    d = (Ut_gpu.double().cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    tol = torch.maximum(1e-12 * scale, 20 * sig)
    return bool((d <= tol).all()), d.tolist(), tol.tolist()


def per_var_rel(a, b, scale=None):
    a, b = a.double().cpu(), b.double().cpu()
    d = (a - b).transpose(0, 1).reshape(5, -1).norm(dim=1)
    s = (b if scale is None else scale).transpose(0, 1).reshape(5, -1).norm(dim=1)
    return (d / s).max().item()


CASES = [
    # (name, mesh kwargs, solver kwargs, state)
    ("tgv_lgl_N3_roe", dict(nelem=(3, 3, 3), reorient_seed=1), dict(N=3, node_type=1, riemann=0), "tgv"),
    ("tgv_lg_N1_hllc", dict(nelem=(3, 3, 3), reorient_seed=2), dict(N=1, riemann=1), "perturbed"),
    ("pert_lg_N2_roe", dict(nelem=(3, 2, 5), reorient_seed=3), dict(N=2, riemann=0), "perturbed"),
    ("pert_lg_N4_hllc", dict(nelem=(2, 3, 2), reorient_seed=4), dict(N=4, riemann=1), "perturbed"),
    ("pert_lg_N5_roesmooth", dict(nelem=(2, 2, 3), reorient_seed=5), dict(N=5, riemann=2, mu=1 / 400.0), "perturbed"),
    ("tgv_lg_N7_hllc", dict(nelem=(2, 2, 3), reorient_seed=6), dict(N=7, riemann=1), "tgv"),
    ("pert_lgl_N6_hllc", dict(nelem=(2, 2, 2), reorient_seed=7), dict(N=6, node_type=1, riemann=1), "perturbed"),
    ("tgv_lgl_N7_hllc", dict(nelem=(2, 2, 3), reorient_seed=7), dict(N=7, node_type=1, riemann=1), "tgv"),
    ("pert_lg_N5_rusanov", dict(nelem=(3, 2, 2), reorient_seed=9), dict(N=5, riemann=3), "perturbed"),
    ("tgv_lgl_N4_rusanov", dict(nelem=(2, 3, 2), reorient_seed=10), dict(N=4, node_type=1, riemann=3), "tgv"),
    ("curved_fs_lg_N4", dict(nelem=(3, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=4, mapping="sine",
                             periodic=(False,) * 3, reorient_seed=8),
     dict(N=4, Ngeo=4, riemann=1, bc_exact=1), "perturbed_small"),
    ("curved_mms_lg_N3", dict(nelem=(2, 3, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=3, mapping="sine",
                              periodic=(False, True, False)),
     dict(N=3, Ngeo=3, riemann=1, bc_exact=2, source=True), "manufactured"),
]


def _state(kind, mesh, N, nt):
    x = mesh.node_coords(N, nt)
    if kind == "tgv":
        return wl.taylor_green(x)
    if kind == "perturbed":
        return wl.perturbed(x, seed=11)
    if kind == "perturbed_small":
        return wl.freestream(x) * (1 + 0.01 * np.sin(3 * x[:, :1]))
    return wl.manufactured(x, 0.0)


@pytest.mark.parametrize("name,mk,sk,state", CASES, ids=[c[0] for c in CASES])
def test_rhs_parity_fp64(name, mk, sk, state):
    mesh = wl.box_mesh(**mk)
    sk = dict(sk, precision=0)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = _state(state, mesh, sk["N"], sk.get("node_type", 0))
    t = 0.1
    Ut = s.rhs(torch.tensor(U0, device=DEV), t)
    ok, d, tol = rhs_parity_ok(Ut, dg, torch.tensor(U0), t, mesh)
    s.close()
    assert ok, (d, tol)


def test_freestream_curved_50_steps():
    """C4a shape (reduced): the free stream stays exact on the curved mesh."""
    N = 7
    mesh = wl.box_mesh((3, 3, 3), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3)
    s = _solver(dict(N=N, Ngeo=N, riemann=1, bc_exact=1), mesh)
    U0 = torch.tensor(wl.freestream(mesh.node_coords(N, 0)), device=DEV)
    U = U0.clone()
    s.run(U, 50, 1e-3)
    err = (U - U0).abs().max().item()
    s.close()
    assert err < 1e-12, err


def test_rk_steps_c1_config():
    """C1: 4^3 periodic, N=3 LGL, Roe, 10 LSERK4(5) steps of dt = 1e-3."""
    mesh = wl.box_mesh((4, 4, 4), Ngeo=1)
    sk = dict(N=3, node_type=1, riemann=0)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = wl.taylor_green(mesh.node_coords(3, 1))
    U = torch.tensor(U0, device=DEV)
    s.run(U, 10, 1e-3)
    ref = dg.run(torch.tensor(U0), 10, 1e-3)
    err = per_var_rel(U, ref)
    s.close()
    assert err < 1e-12, err


def test_rk_steps_stages_and_reorientation():
    """rk_step_stages stores the five stage inputs; reoriented frames, N=5."""
    mesh = wl.box_mesh((3, 2, 2), Ngeo=1, reorient_seed=12)
    sk = dict(N=5, riemann=1)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = wl.perturbed(mesh.node_coords(5, 0), seed=4)
    U = torch.tensor(U0, device=DEV)
    dU = torch.zeros_like(U)
    stages = torch.empty((5,) + U.shape, dtype=U.dtype, device=DEV)
    s.step_stages(U, dU, 0.0, 2e-3, stages)
    st_ref = []
    Ur, dUr = dg.rk_step(torch.tensor(U0), torch.zeros_like(torch.tensor(U0)), 0.0, 2e-3, stages_out=st_ref)
    assert per_var_rel(U, Ur) < 1e-12
    assert per_var_rel(dU, dUr) < 1e-11
    for k in range(5):
        assert per_var_rel(stages[k], st_ref[k]) < 1e-12
    s.close()


def test_c2_full_size_rhs_and_invariants():
    """C2 at full size (16^3, N=7 Gauss, HLLC): one RHS against the oracle, then
    100 steps with conservation of mass, momentum and energy and decaying KE."""
    N = 7
    mesh = wl.box_mesh((16, 16, 16), Ngeo=1)
    sk = dict(N=N, riemann=1)
    s = _solver(sk, mesh)
    U0 = wl.taylor_green(mesh.node_coords(N, 0))
    U = torch.tensor(U0, device=DEV)
    Ut = s.rhs(U, 0.0)
    dg = _oracle(sk, mesh)
    ok, d, tol = rhs_parity_ok(Ut, dg, torch.tensor(U0), 0.0, mesh)
    assert ok, (d, tol)
    r0 = s.reduce(U)
    o_int = dg.integrals(torch.tensor(U0))
    assert abs(r0["kinetic_energy"] - float(o_int[5])) < 1e-12 * abs(float(o_int[5]))
    assert abs(r0["dt_max"] - dg.dt_max(torch.tensor(U0), 0.9)) < 1e-12 * r0["dt_max"]
    dt = r0["dt_max"]
    del dg
    s.run(U, 100, dt)
    r1 = s.reduce(U)
    for key in ("mass", "mom_x", "mom_y", "mom_z", "energy"):
        assert abs(r1[key] - r0[key]) < 1e-12 * max(1.0, abs(r0["energy"])), key
    assert r1["kinetic_energy"] < r0["kinetic_energy"]
    s.close()


def test_reduce_matches_oracle():
    mesh = wl.box_mesh((3, 3, 2), Ngeo=1, reorient_seed=3)
    sk = dict(N=4, riemann=1)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = wl.perturbed(mesh.node_coords(4, 0), seed=8)
    U = torch.tensor(U0, device=DEV)
    Ut = s.rhs(U)
    r = s.reduce(U, Ut, cfl=0.5)
    ints = dg.integrals(torch.tensor(U0))
    for q, key in enumerate(["mass", "mom_x", "mom_y", "mom_z", "energy", "kinetic_energy"]):
        assert abs(r[key] - float(ints[q])) < 1e-12 * max(1.0, abs(float(ints[q]))), key
    Ut_ref = dg.rhs(torch.tensor(U0))
    with torch.enable_grad():
        Ux = torch.tensor(U0).requires_grad_(True)
        (gk,) = torch.autograd.grad(dg.kinetic_energy(Ux), Ux)
    dkedt = float((gk * Ut_ref).sum())
    assert abs(r["dkedt"] - dkedt) < 1e-10 * max(1.0, abs(dkedt))
    assert abs(r["dt_max"] - dg.dt_max(torch.tensor(U0), 0.5, 0.5)) < 1e-13 * r["dt_max"]
    s.close()


def test_run_host_matches_device_path():
    """flexi_rk_run_host, flexi_rk_run (graph replay) and separate flexi_rk_step calls
    give the same bits (the first two hand the face states from step to step through
    the last stage, the third prolongs U at every step)."""
    mesh = wl.box_mesh((3, 3, 3), Ngeo=1)
    sk = dict(N=3, riemann=1)
    s = _solver(sk, mesh)
    U0 = torch.tensor(wl.taylor_green(mesh.node_coords(3, 0)))
    Uh = U0.clone().pin_memory()
    from paper_1910_02858_gb300 import flexi as F

    F.flexi_rk_run_host(s.ctx, Uh, 3, 0.0, 1e-3, torch.cuda.current_stream())
    Ud = U0.to(DEV)
    s.run(Ud, 3, 1e-3)
    Ue = U0.to(DEV)
    s.run(Ue, 3, 1e-3, graph=False)
    torch.cuda.synchronize()
    assert torch.equal(Uh, Ud.cpu())
    assert torch.equal(Ud, Ue)
    s.close()


def test_nonphysical_state_reported():
    from paper_1910_02858_gb300 import flexi as F

    mesh = wl.box_mesh((2, 2, 2), Ngeo=1)
    s = _solver(dict(N=2, riemann=1), mesh)
    U0 = wl.taylor_green(mesh.node_coords(2, 0))
    U0[3, 0] = -1.0  # negative density in one element (host-side injection)
    U = torch.tensor(U0, device=DEV)
    s.rhs(U)
    r = s.reduce(torch.tensor(wl.taylor_green(mesh.node_coords(2, 0)), device=DEV), allow_nonphysical=True)
    assert r["status"] == F.FLEXI_ENONPHYSICAL
    assert s.query(F.Q_STATUS) == 0  # cleared by the report
    s.close()


def test_mesh_errors():
    from paper_1910_02858_gb300 import flexi as F

    mesh = wl.box_mesh((2, 2, 2), Ngeo=1)
    conn = mesh.conn.copy()
    conn[0, 1, 2] = (conn[0, 1, 2] + 1) % 8  # orientation not the inverse of the neighbour's
    with pytest.raises(F.FlexiError) as ei:
        _solver(dict(N=2), wl.BoxMesh(**{**mesh.__dict__, "conn": conn}))
    assert ei.value.code == F.FLEXI_EMESH
    coords = mesh.coords.copy()
    coords[0] = coords[0][:, :, ::-1]  # mirrored element: J < 0
    with pytest.raises(F.FlexiError) as ei:
        _solver(dict(N=2), wl.BoxMesh(**{**mesh.__dict__, "coords": coords}))
    assert ei.value.code == F.FLEXI_EMESH
    with pytest.raises(F.FlexiError) as ei:
        _solver(dict(N=8), mesh)
    assert ei.value.code == F.FLEXI_EUNSUPPORTED


def test_kernel_timing_hooks():
    from paper_1910_02858_gb300 import flexi as F

    mesh = wl.box_mesh((4, 4, 4), Ngeo=1)
    s = _solver(dict(N=3), mesh)
    U = torch.tensor(wl.taylor_green(mesh.node_coords(3, 0)), device=DEV)
    F.flexi_profile(s.ctx, True)
    s.run(U, 2, 1e-3)
    t = F.flexi_kernel_times(s.ctx)
    # one prolongation: the second step takes its face states from the first step's last stage;
    # with fewer elements than SMs (FP64, n = 4, BR1) k_surf_face computes the face fluxes
    fused = mesh.K < torch.cuda.get_device_properties(0).multi_processor_count
    assert t["lift_vol"][1] == 10 and t["surf_rk"][1] == 10 and t["prolong"][1] == 1
    assert t["face"][1] == (0 if fused else 10)
    assert all(v[0] >= 0 for v in t.values())
    s.close()


@pytest.mark.parametrize("mk,sk", [
    (dict(nelem=(4, 4, 4), Ngeo=1), dict(N=3, node_type=1, riemann=0)),  # C1
    (dict(nelem=(2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=2, mapping="sine", periodic=(False,) * 3,
          reorient_seed=3), dict(N=4, Ngeo=2, riemann=1, bc_exact=1)),
    (dict(nelem=(2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, periodic=(False, True, True)),
     dict(N=3, riemann=1, bc_exact=2, source=True)),  # time-dependent: eager path
])
def test_graph_run_matches_eager_steps(mk, sk):
    """flexi_rk_run (one eager step, then CUDA-graph replay of one step when the
    operator does not depend on t) gives bit-identical states to launching every
    step, also on a second call that reuses the captured graph."""
    mesh = wl.box_mesh(**mk)
    s = _solver(sk, mesh)
    U0 = _state("perturbed_small" if sk.get("bc_exact") == 1 else "tgv", mesh, sk["N"], sk.get("node_type", 0))
    Ua = torch.tensor(U0, device=DEV)
    Ub = Ua.clone()
    s.run(Ua, 7, 1e-3, graph=True)
    s.run(Ua, 5, 1e-3, t0=7e-3, graph=True)
    s.run(Ub, 7, 1e-3, graph=False)
    s.run(Ub, 5, 1e-3, t0=7e-3, graph=False)
    torch.cuda.synchronize()
    s.close()
    assert torch.equal(Ua, Ub)
