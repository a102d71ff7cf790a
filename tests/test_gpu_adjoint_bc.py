"""Discrete adjoint of the CUDA path on meshes with boundaries (exact-state,
outflow and slip-wall sides; the manufactured source term), with the HLLC,
Rusanov and entropy-conservative fluxes (reversed by dual numbers) and with BR2
face gradients or the split-form volume integral (KEP / EC two-point fluxes),
against the oracle's reverse-mode derivative and central finite-difference
dot-product tests."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.dgsem import DGSEM, EC, HLLC, ROE, RUSANOV, Params

RIEM = {0: ROE, 1: HLLC, 2: ROE, 3: RUSANOV, 4: EC}

from test_gpu_parity import DEV

pytestmark = pytest.mark.gpu

CASES = [
    # (name, mesh kwargs, N, node_type, riemann (0 Roe, 1 HLLC, 2 smoothed Roe, 3 Rusanov, 4 EC),
    #  bc_exact, source, kinds)
    ("mixed_lg_N3_smooth", dict(nelem=(2, 3, 2), Ngeo=3, mapping="sine", reorient_seed=4,
                                bc_ids=[0, 1, 2, 2, 2, 2]), 3, 0, 2, 1, False, {1: 1, 2: 2}),
    ("slip_box_lgl_N4_roe", dict(nelem=(2, 2, 2), Ngeo=2, mapping="sine", reorient_seed=2, bc_ids=[2] * 6),
     4, 1, 0, 1, False, {2: 2}),
    ("manufactured_lg_N2_exact_outflow", dict(nelem=(3, 2, 2), Ngeo=2, mapping="sine", reorient_seed=1,
                                              bc_ids=[0, 1, 0, 0, 1, 1]), 2, 0, 2, 2, True, {1: 1}),
    ("in_out_periodic_yz_N5", dict(nelem=(3, 2, 2), periodic=(False, True, True), reorient_seed=3,
                                   bc_ids=[0, 1, 0, 0, 0, 0]), 5, 0, 2, 1, False, {1: 1}),
    ("hllc_mixed_lg_N3", dict(nelem=(2, 3, 2), Ngeo=3, mapping="sine", reorient_seed=4,
                              bc_ids=[0, 1, 2, 2, 2, 2]), 3, 0, 1, 1, False, {1: 1, 2: 2}),
    ("hllc_periodic_lg_N4", dict(nelem=(2, 2, 3), periodic=(True,) * 3, reorient_seed=5), 4, 0, 1, 1, False, {}),
    ("rusanov_slip_lgl_N3", dict(nelem=(2, 2, 2), Ngeo=2, mapping="sine", reorient_seed=2, bc_ids=[2] * 6),
     3, 1, 3, 1, False, {2: 2}),
    ("ec_periodic_lgl_N3", dict(nelem=(2, 3, 2), periodic=(True,) * 3, reorient_seed=6), 3, 1, 4, 1, False, {}),
    ("hllc_manufactured_N2", dict(nelem=(3, 2, 2), Ngeo=2, mapping="sine", reorient_seed=1,
                                  bc_ids=[0, 1, 0, 0, 1, 1]), 2, 0, 1, 2, True, {1: 1}),
]


def _pair(case, eta=None, split=0):
    """GPU solver and oracle for a case; eta given: BR2 lifting with that penalty;
    split 1 / 2: the kinetic-energy-preserving / entropy-conservative split form."""
    from paper_1910_02858_gb300 import Solver, SolverConfig

    name, mk, N, nt, riem, bc_exact, source, kinds = case
    mk = dict(dict(lo=(-1,) * 3, hi=(1,) * 3, periodic=(False,) * 3), **mk)
    mesh = wl.box_mesh(**mk)
    lift = {} if eta is None else dict(lifting=1, eta_br2=eta)
    if split:
        lift["split_form"] = split
    s = Solver(SolverConfig(N=N, Ngeo=mk.get("Ngeo", 1), node_type=nt, riemann=riem, mu=1 / 400.0,
                            bc_exact=bc_exact, source=source, adjoint=True, **lift), mesh.coords, mesh.conn,
               device=DEV)
    for bc_id, kind in kinds.items():
        s.set_bc(bc_id, kind)
    olift = {} if eta is None else dict(lifting="br2", eta_br2=eta)
    if split:
        olift["split"] = {1: "pirozzoli", 2: "chandrashekar"}[split]
    dg = DGSEM(Params(N=N, node_type=nt, riemann=RIEM[riem], smooth_roe=riem == 2, mu=1 / 400.0, bc_exact=bc_exact,
                      source=source, bc_kinds=dict(kinds), **olift), mesh.coords, mesh.conn)
    U0 = wl.perturbed(np.pi * mesh.node_coords(N, nt), seed=7)
    return s, dg, U0


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_rhs_adjoint_with_boundaries_vs_oracle(case):
    s, dg, U0 = _pair(case)
    lam = np.random.default_rng(3).normal(size=U0.shape)
    out = s.rhs_adjoint(torch.tensor(U0, device=DEV), torch.tensor(lam, device=DEV), 0.3)
    ref = dg.rhs_vjp(torch.tensor(U0), 0.3, torch.tensor(lam))
    s.close()
    d = (out.cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    r = ref.transpose(0, 1).reshape(5, -1).norm(dim=1)
    assert float((d / r).max()) < 1e-10, (d / r).tolist()


@pytest.mark.parametrize("ci", [2, 8], ids=[CASES[2][0], CASES[8][0]])
def test_adjoint_step_with_boundaries_vs_oracle(ci):
    """One reverse LSERK4(5) step from t = 0.2: the exact-state sides and the source
    are taken at the stage times of the forward step."""
    s, dg, U0 = _pair(CASES[ci])
    rng = np.random.default_rng(9)
    lamU0, lamdU0 = rng.normal(size=U0.shape), rng.normal(size=U0.shape)
    t0, dt = 0.2, 1e-3
    U = torch.tensor(U0, device=DEV)
    stages = torch.empty((5,) + U.shape, dtype=U.dtype, device=DEV)
    s.step_stages(U, torch.zeros_like(U), t0, dt, stages)
    lamU, lamdU = torch.tensor(lamU0, device=DEV), torch.tensor(lamdU0, device=DEV)
    s.adjoint_step(stages, lamU, lamdU, t0, dt)
    st_ref = []
    dg.rk_step(torch.tensor(U0), torch.zeros_like(torch.tensor(U0)), t0, dt, stages_out=st_ref)
    rU, _ = dg.adjoint_step(st_ref, torch.tensor(lamU0), torch.tensor(lamdU0), t0, dt)
    s.close()
    assert float((lamU.cpu() - rU).norm() / rU.norm()) < 1e-12


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[4], CASES[6]],
                         ids=[CASES[0][0], CASES[1][0], CASES[4][0], CASES[6][0]])
def test_dot_product_with_finite_difference_jvp_boundaries(case):
    """<lam, J v> from a central difference of flexi_rhs equals <J^T lam, v>, with
    no oracle involved."""
    s, _, U0 = _pair(case)
    U0 = torch.tensor(U0, device=DEV)
    g = torch.Generator(device="cpu").manual_seed(5)
    v = torch.randn(U0.shape, generator=g, dtype=torch.float64).to(DEV)
    lam = torch.randn(U0.shape, generator=g, dtype=torch.float64).to(DEV)
    eps = 1e-6
    Jv = (s.rhs(U0 + eps * v, 0.1) - s.rhs(U0 - eps * v, 0.1)) / (2 * eps)
    a = float((lam * Jv).sum())
    b = float((s.rhs_adjoint(U0, lam, 0.1) * v).sum())
    s.close()
    assert abs(a - b) < 1e-6 * abs(b), (a, b)


def test_adjoint_with_boundaries_fp32_vs_fp64():
    """The FP32 form's adjoint on a mesh with boundaries against the FP64 one."""
    from paper_1910_02858_gb300 import Solver, SolverConfig

    s64, _, U0 = _pair(CASES[0])
    name, mk, N, nt, riem, bc_exact, source, kinds = CASES[0]
    mesh = wl.box_mesh(**dict(dict(lo=(-1,) * 3, hi=(1,) * 3, periodic=(False,) * 3), **mk))
    s32 = Solver(SolverConfig(N=N, Ngeo=mk["Ngeo"], riemann=riem, mu=1 / 400.0, bc_exact=bc_exact, precision=1,
                              adjoint=True), mesh.coords, mesh.conn, device=DEV)
    for bc_id, kind in kinds.items():
        s32.set_bc(bc_id, kind)
    lam = np.random.default_rng(3).normal(size=U0.shape)
    a = s64.rhs_adjoint(torch.tensor(U0, device=DEV), torch.tensor(lam, device=DEV), 0.0).cpu()
    b = s32.rhs_adjoint(torch.tensor(U0, device=DEV, dtype=torch.float32),
                        torch.tensor(lam, device=DEV, dtype=torch.float32), 0.0).double().cpu()
    s64.close()
    s32.close()
    d = (a - b).transpose(0, 1).reshape(5, -1).norm(dim=1)
    r = a.transpose(0, 1).reshape(5, -1).norm(dim=1)
    assert float((d / r).max()) < 1e-4, (d / r).tolist()


BR2_CASES = [  # (case, eta)
    (CASES[0], 2.0), (CASES[1], 2.0), (CASES[2], 0.0), (CASES[4], 5.0), (CASES[6], 2.0),
]


@pytest.mark.parametrize("case,eta", BR2_CASES, ids=[f"br2_{c[0]}_eta{e:g}" for c, e in BR2_CASES])
def test_rhs_adjoint_br2_vs_oracle(case, eta):
    """BR2 face gradients (broken gradient plus eta times the face's own lifting):
    the reverse of the jumps reaches U* and the element's own face state."""
    s, dg, U0 = _pair(case, eta)
    lam = np.random.default_rng(4).normal(size=U0.shape)
    out = s.rhs_adjoint(torch.tensor(U0, device=DEV), torch.tensor(lam, device=DEV), 0.3)
    ref = dg.rhs_vjp(torch.tensor(U0), 0.3, torch.tensor(lam))
    s.close()
    d = (out.cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    r = ref.transpose(0, 1).reshape(5, -1).norm(dim=1)
    assert float((d / r).max()) < 1e-10, (d / r).tolist()


def test_br2_adjoint_dot_product_and_step():
    """BR2 without the oracle: central-difference dot-product test; and one reverse
    LSERK4(5) step against the oracle."""
    s, dg, U0 = _pair(CASES[0], 2.0)
    Ud = torch.tensor(U0, device=DEV)
    g = torch.Generator(device="cpu").manual_seed(6)
    v = torch.randn(Ud.shape, generator=g, dtype=torch.float64).to(DEV)
    lam = torch.randn(Ud.shape, generator=g, dtype=torch.float64).to(DEV)
    eps = 1e-6
    Jv = (s.rhs(Ud + eps * v, 0.1) - s.rhs(Ud - eps * v, 0.1)) / (2 * eps)
    a = float((lam * Jv).sum())
    b = float((s.rhs_adjoint(Ud, lam, 0.1) * v).sum())
    assert abs(a - b) < 1e-6 * abs(b), (a, b)
    rng = np.random.default_rng(11)
    lamU0, lamdU0 = rng.normal(size=U0.shape), rng.normal(size=U0.shape)
    stages = torch.empty((5,) + Ud.shape, dtype=Ud.dtype, device=DEV)
    s.step_stages(Ud.clone(), torch.zeros_like(Ud), 0.2, 1e-3, stages)
    lamU, lamdU = torch.tensor(lamU0, device=DEV), torch.tensor(lamdU0, device=DEV)
    s.adjoint_step(stages, lamU, lamdU, 0.2, 1e-3)
    st_ref = []
    dg.rk_step(torch.tensor(U0), torch.zeros_like(torch.tensor(U0)), 0.2, 1e-3, stages_out=st_ref)
    rU, _ = dg.adjoint_step(st_ref, torch.tensor(lamU0), torch.tensor(lamdU0), 0.2, 1e-3)
    s.close()
    assert float((lamU.cpu() - rU).norm() / rU.norm()) < 1e-12


SPLIT_CASES = [  # Gauss-Lobatto cases (the split form is built on LGL nodes) x split form
    (CASES[1], 1), (CASES[1], 2), (CASES[6], 1), (CASES[7], 2),
    (("kep_periodic_lgl_N4_hllc", dict(nelem=(2, 3, 2), periodic=(True,) * 3, reorient_seed=8), 4, 1, 1, 1, False,
      {}), 1),
    (("kep_curved_lgl_N3_roe_bc", dict(nelem=(2, 2, 3), Ngeo=3, mapping="sine", reorient_seed=9,
                                       bc_ids=[0, 1, 2, 2, 1, 0]), 3, 1, 2, 1, False, {1: 1, 2: 2}), 1),
]


@pytest.mark.parametrize("case,split", SPLIT_CASES, ids=[f"split{sp}_{c[0]}" for c, sp in SPLIT_CASES])
def test_rhs_adjoint_split_form_vs_oracle(case, split):
    s, dg, U0 = _pair(case, split=split)
    lam = np.random.default_rng(5).normal(size=U0.shape)
    out = s.rhs_adjoint(torch.tensor(U0, device=DEV), torch.tensor(lam, device=DEV), 0.3)
    ref = dg.rhs_vjp(torch.tensor(U0), 0.3, torch.tensor(lam))
    s.close()
    d = (out.cpu() - ref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    r = ref.transpose(0, 1).reshape(5, -1).norm(dim=1)
    assert float((d / r).max()) < 1e-10, (d / r).tolist()


@pytest.mark.parametrize("split", [1, 2])
def test_split_form_adjoint_dot_product(split):
    """Central-difference dot-product test of the split-form adjoint (no oracle)."""
    s, _, U0 = _pair(CASES[1], split=split)
    Ud = torch.tensor(U0, device=DEV)
    g = torch.Generator(device="cpu").manual_seed(7)
    v = torch.randn(Ud.shape, generator=g, dtype=torch.float64).to(DEV)
    lam = torch.randn(Ud.shape, generator=g, dtype=torch.float64).to(DEV)
    eps = 1e-6
    Jv = (s.rhs(Ud + eps * v, 0.1) - s.rhs(Ud - eps * v, 0.1)) / (2 * eps)
    a = float((lam * Jv).sum())
    b = float((s.rhs_adjoint(Ud, lam, 0.1) * v).sum())
    s.close()
    assert abs(a - b) < 1e-6 * abs(b), (a, b)
