"""BR2 face gradients on the GPU (flexi_params.lifting = FLEXI_LIFTING_BR2) through
the C ABI against the oracle's BR2 reading.

Right-hand sides use the rounding-sensitivity tolerance of test_gpu_parity (1-ulp
noise on the state and on the mesh coordinates, 20 sigma; FP32 scaled by 2^29);
states after time steps 1e-12 relative L2 per conserved variable (FP64)."""
import numpy as np
import pytest
import torch

import workloads as wl

from test_gpu_parity import DEV, _oracle, _solver, _state, per_var_rel, rhs_parity_ok, rounding_sensitivity

pytestmark = pytest.mark.gpu

CASES = [
    # (name, mesh kwargs, solver kwargs, state)
    ("lg_N3_hllc_eta2", dict(nelem=(3, 2, 2), reorient_seed=1), dict(N=3, riemann=1, mu=0.01), "perturbed"),
    ("lgl_N4_roe_eta2", dict(nelem=(2, 3, 2), reorient_seed=2), dict(N=4, node_type=1, riemann=0, mu=0.01),
     "perturbed"),
    ("lg_N7_hllc_eta0", dict(nelem=(2, 2, 3), reorient_seed=3), dict(N=7, riemann=1, eta_br2=0.0), "tgv"),
    ("lgl_N6_rusanov_eta5", dict(nelem=(2, 2, 2), reorient_seed=4), dict(N=6, node_type=1, riemann=3, eta_br2=5.0,
                                                                         mu=0.01), "perturbed"),
    ("lg_N1_hllc", dict(nelem=(3, 3, 3), reorient_seed=5), dict(N=1, riemann=1, mu=0.01), "perturbed"),
    ("curved_mms_lg_N3", dict(nelem=(2, 3, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=3, mapping="sine",
                              periodic=(False, True, False)),
     dict(N=3, Ngeo=3, riemann=1, bc_exact=2, source=True, mu=0.02), "manufactured"),
]


@pytest.mark.parametrize("name,mk,sk,state", CASES, ids=[c[0] for c in CASES])
def test_br2_rhs_parity_fp64(name, mk, sk, state):
    mesh = wl.box_mesh(**mk)
    sk = dict(sk, lifting=1, precision=0)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = _state(state, mesh, sk["N"], sk.get("node_type", 0))
    Ut = s.rhs(torch.tensor(U0, device=DEV), 0.1)
    ok, d, tol = rhs_parity_ok(Ut, dg, torch.tensor(U0), 0.1, mesh)
    s.close()
    assert ok, (d, tol)


@pytest.mark.parametrize("N,nt", [(7, 0), (4, 1)])
def test_br2_rhs_parity_fp32(N, nt):
    mesh = wl.box_mesh((3, 2, 2), reorient_seed=N)
    sk = dict(N=N, node_type=nt, riemann=1, mu=0.01, lifting=1, precision=1)
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


def test_br2_differs_from_br1_on_gpu():
    mesh = wl.box_mesh((2, 2, 2), reorient_seed=3)
    U0 = torch.tensor(wl.perturbed(mesh.node_coords(3, 0), seed=5), device=DEV)
    a = _solver(dict(N=3, riemann=1, mu=0.01), mesh)
    b = _solver(dict(N=3, riemann=1, mu=0.01, lifting=1), mesh)
    ra, rb = a.rhs(U0), b.rhs(U0)
    a.close()
    b.close()
    assert (ra - rb).abs().max().item() > 1e-8 * ra.abs().max().item()


def test_br2_rk_steps_match_oracle():
    mesh = wl.box_mesh((4, 4, 4), Ngeo=1, reorient_seed=2)
    sk = dict(N=3, riemann=1, mu=0.01, lifting=1)
    s = _solver(sk, mesh)
    dg = _oracle(sk, mesh)
    U0 = wl.taylor_green(mesh.node_coords(3, 0))
    U = torch.tensor(U0, device=DEV)
    s.run(U, 20, 2e-3)
    Ur = dg.run(torch.tensor(U0), 20, 2e-3)
    err = per_var_rel(U, Ur)
    s.close()
    assert err < 1e-12, err


def test_br2_with_mortars_matches_oracle():
    from oracle.dgsem import DGSEM, HLLC, Params
    from paper_1910_02858_gb300 import Solver, SolverConfig

    mesh = wl.mortar_box_mesh(refine=(2, 2, 2), ny=1, nz=1, reorient_seed=3)
    s = Solver(SolverConfig(N=3, riemann=1, mu=0.01, lifting=1), mesh.coords, mesh.conn, device=DEV,
               mortars=mesh.mortars)
    dg = DGSEM(Params(N=3, riemann=HLLC, mu=0.01, lifting="br2"), mesh.coords, mesh.conn, mesh.mortars)
    from test_gpu_mortar import _check_rhs

    U0 = wl.perturbed(np.pi * mesh.node_coords(3, 0), seed=11)
    Ut = s.rhs(torch.tensor(U0, device=DEV), 0.0)
    ok, d, tol = _check_rhs(Ut, dg, torch.tensor(U0), 0.0, mesh)
    s.close()
    assert ok, (d, tol)


def test_br2_unsupported_and_invalid():
    from paper_1910_02858_gb300 import flexi as F

    mesh = wl.box_mesh((2, 2, 2))
    for kw, code in ((dict(N=3, lifting=1, precision=2), F.FLEXI_EUNSUPPORTED),
                     (dict(N=3, node_type=1, lifting=1, split_form=1), F.FLEXI_EUNSUPPORTED),
                     (dict(N=3, lifting=2), F.FLEXI_EINVAL), (dict(N=3, lifting=1, eta_br2=-1.0), F.FLEXI_EINVAL)):
        with pytest.raises(F.FlexiError) as ei:
            _solver(kw, mesh)
        assert ei.value.code == code
