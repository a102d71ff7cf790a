"""State parity of the headline path after LSERK4(5) time steps at N = 7.

The path: N = 7, HLLC, BR1, FP64, Taylor-Green vortex (Re 1600, Ma 0.1), step
size from CFL 0.9 (Sec. 3.1 Eq. semiDiscrete, Sec. 3.4, Eqs. CFLCondition and
DFLCondition).  The CUDA path's state after ten steps is compared with the
oracle's, variable by variable, in relative L2:

    ||U_gpu,v - U_oracle,v|| / ||U_oracle,v|| <= 1e-12

with the three momentum components measured against the norm of the whole
momentum vector (the Taylor-Green w-momentum starts at exactly zero, so its own
norm is no scale).  This exercises the n = 8 instances of the lifting/volume
kernel and of the surface kernel with its fused RK update over whole steps.

Gauss-Lobatto nodes: the low-Mach state carries a large constant pressure
(p0 = 71.4), which the face terms multiply by l_hat(+-1) = N(N+1)/2 = 28, so a
rounding difference in the metric terms (the two implementations compute them
from the node coordinates with their own summation orders) becomes a force that
the time steps integrate.  There the test also measures the oracle's own change
under 1-ulp relative noise on the node coordinates and accepts
max(1e-12, 2 x that change); both numbers are printed.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle.dgsem import DGSEM, HLLC, Params

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_02858_gb300 import build as b

    b.build()
    from paper_1910_02858_gb300 import flexi as F

    F.lib()


def rel_per_var(U, Uref):
    """Relative L2 per conserved variable; momentum against the momentum-vector norm."""
    U, Uref = U.double().cpu(), Uref.double().cpu()
    d = (U - Uref).transpose(0, 1).reshape(5, -1).norm(dim=1)
    r = Uref.transpose(0, 1).reshape(5, -1).norm(dim=1)
    r[1:4] = Uref[:, 1:4].norm()
    return (d / r).tolist()


def coordinate_rounding_floor(mesh, N, node_type, U0, nsteps, dt, ref, trials=2):
    """Largest relative change (rel_per_var) of the oracle's state after nsteps
    under random 1-ulp relative perturbations of the mesh node coordinates."""
    rng = np.random.default_rng(4321)
    floor = 0.0
    for _ in range(trials):
        coords = mesh.coords * (1 + 2.2e-16 * (2 * rng.random(mesh.coords.shape) - 1))
        dgx = DGSEM(Params(N=N, node_type=node_type, riemann=HLLC), coords, mesh.conn)
        floor = max(floor, max(rel_per_var(dgx.run(torch.tensor(U0), nsteps, dt), ref)))
    return floor


def _run_both(mesh, N, node_type, U0, nsteps):
    from paper_1910_02858_gb300 import Solver, SolverConfig

    dg = DGSEM(Params(N=N, node_type=node_type, riemann=HLLC), mesh.coords, mesh.conn)
    dt = dg.dt_max(torch.tensor(U0), 0.9)
    s = Solver(SolverConfig(N=N, node_type=node_type, riemann=1), mesh.coords, mesh.conn, device=DEV)
    try:
        assert abs(s.reduce(torch.tensor(U0, device=DEV))["dt_max"] - dt) < 1e-13 * dt
        U = torch.tensor(U0, device=DEV)
        s.run(U, nsteps, dt)
        torch.cuda.synchronize()
        Ug = U.cpu()
    finally:
        s.close()
    ref = dg.run(torch.tensor(U0), nsteps, dt)
    return Ug, ref, dt


CASES = [
    ("tgv_lg_2x2x3", (2, 2, 3), 6, 0, "tgv"),
    ("tgv_lgl_2x2x3", (2, 2, 3), 7, 1, "tgv"),
    ("perturbed_lg_3x2x2", (3, 2, 2), 13, 0, "perturbed"),
]


@pytest.mark.parametrize("name,nelem,seed,nt,state", CASES, ids=[c[0] for c in CASES])
def test_n7_ten_steps_small_mesh(name, nelem, seed, nt, state):
    N = 7
    mesh = wl.box_mesh(nelem, Ngeo=1, reorient_seed=seed)
    x = mesh.node_coords(N, nt)
    U0 = wl.taylor_green(x) if state == "tgv" else wl.perturbed(x, seed=21)
    Ug, ref, dt = _run_both(mesh, N, nt, U0, 10)
    err = rel_per_var(Ug, ref)
    tol = TOL
    if nt == 1:
        floor = coordinate_rounding_floor(mesh, N, nt, U0, 10, dt, ref)
        tol = max(TOL, 2 * floor)
        print(name, "oracle change under 1-ulp coordinate noise %.2e" % floor)
    print(name, "dt", dt, "rel L2 per variable", ["%.2e" % e for e in err], "tolerance %.2e" % tol)
    assert max(err) <= tol, (err, tol)


def test_c2_full_size_ten_steps():
    """The full headline workload: 16^3 elements, N = 7 Gauss, 2,097,152 DOF."""
    N = 7
    mesh = wl.box_mesh((16, 16, 16), Ngeo=1)
    U0 = wl.taylor_green(mesh.node_coords(N, 0))
    Ug, ref, dt = _run_both(mesh, N, 0, U0, 10)
    err = rel_per_var(Ug, ref)
    print("c2 16^3 dt", dt, "rel L2 per variable", ["%.2e" % e for e in err])
    assert max(err) <= TOL, err


def test_n5_ten_steps_precision_form_order():
    """N = 5, the order of the precision form's 32^3 workload, whose FP32 errors are
    measured against this FP64 path: Taylor-Green on a reoriented 3x2x2 Gauss mesh (the
    n = 6 kernel instances), ten steps at CFL 0.9, 1e-12 per conserved variable."""
    N = 5
    mesh = wl.box_mesh((3, 2, 2), Ngeo=1, reorient_seed=9)
    U0 = wl.taylor_green(mesh.node_coords(N, 0))
    Ug, ref, dt = _run_both(mesh, N, 0, U0, 10)
    err = rel_per_var(Ug, ref)
    print("N5 tgv_lg_3x2x2 dt", dt, "rel L2 per variable", ["%.2e" % e for e in err])
    assert max(err) <= TOL, err


def _run_variant(mesh, sk, pk, U0, nsteps, mortars=None):
    """The CUDA path (SolverConfig sk) and the oracle (Params pk) over nsteps steps at
    the oracle's CFL-0.9 step size; returns both states, the step and the oracle."""
    from paper_1910_02858_gb300 import Solver, SolverConfig

    dg = DGSEM(Params(**pk), mesh.coords, mesh.conn, mortars)
    dt = dg.dt_max(torch.tensor(U0), 0.9)
    s = Solver(SolverConfig(**sk), mesh.coords, mesh.conn, device=DEV, mortars=mortars)
    try:
        U = torch.tensor(U0, device=DEV)
        s.run(U, nsteps, dt)
        torch.cuda.synchronize()
        Ug = U.cpu()
    finally:
        s.close()
    return Ug, dg.run(torch.tensor(U0), nsteps, dt), dt, dg


VARIANTS = [
    # (name, mesh, solver kwargs, oracle kwargs)
    ("split_kep_lgl_2x2x3", lambda: wl.box_mesh((2, 2, 3), Ngeo=1, reorient_seed=11),
     dict(N=7, node_type=1, riemann=1, split_form=1), dict(N=7, node_type=1, riemann=HLLC, split="pirozzoli")),
    ("br2_lg_2x2x3", lambda: wl.box_mesh((2, 2, 3), Ngeo=1, reorient_seed=12),
     dict(N=7, riemann=1, lifting=1, eta_br2=2.0), dict(N=7, riemann=HLLC, lifting="br2", eta_br2=2.0)),
    ("mortar_type3_lg", lambda: wl.mortar_box_mesh(nx=1, ny=1, nz=1, refine=(1, 2, 2), lo=(0.0,) * 3,
                                                   hi=(2 * np.pi,) * 3, reorient_seed=4),
     dict(N=7, riemann=1), dict(N=7, riemann=HLLC)),
]


@pytest.mark.parametrize("name,make_mesh,sk,pk", VARIANTS, ids=[v[0] for v in VARIANTS])
def test_n7_ten_steps_variant_forms(name, make_mesh, sk, pk):
    """The split-form volume integral (kinetic-energy preserving, Gauss-Lobatto), BR2
    lifting and a mesh with type-3 mortars at N = 7: ten steps against the oracle on a
    perturbed (Ma 0.3) state; Gauss-Lobatto with the coordinate-rounding floor above."""
    mesh = make_mesh()
    mortars = getattr(mesh, "mortars", None)
    nt = sk.get("node_type", 0)
    U0 = wl.perturbed(mesh.node_coords(7, nt), seed=23)
    Ug, ref, dt, dg = _run_variant(mesh, sk, pk, U0, 10, mortars)
    err = rel_per_var(Ug, ref)
    tol = TOL
    if nt == 1:
        rng = np.random.default_rng(4321)
        floor = 0.0
        for _ in range(2):
            coords = mesh.coords * (1 + 2.2e-16 * (2 * rng.random(mesh.coords.shape) - 1))
            dgx = DGSEM(dg.p, coords, mesh.conn, mortars)
            floor = max(floor, max(rel_per_var(dgx.run(torch.tensor(U0), 10, dt), ref)))
        tol = max(TOL, 2 * floor)
        print(name, "oracle change under 1-ulp coordinate noise %.2e" % floor)
    print(name, "dt", dt, "rel L2 per variable", ["%.2e" % e for e in err], "tolerance %.2e" % tol)
    assert max(err) <= tol, (err, tol)
