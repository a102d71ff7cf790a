"""Pins of the oracle's boundary kinds (Sec. 2.2: boundary conditions imposed
weakly through the outer state of the numerical flux): exact (Dirichlet), outflow
(extrapolated inner state) and slip wall (inner state with the normal velocity
reversed)."""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import equations as eq
from oracle.dgsem import BC_EXACT, BC_OUTFLOW, BC_SLIP_WALL, DGSEM, HLLC, ROE, RUSANOV, Params


def T(a):
    return torch.tensor(a, dtype=torch.float64)


def _mirror_state(x):
    """Even in x (rho, v, w, p) and odd in x (u) about x = 0 and x = pi."""
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    rho = 1.0 + 0.1 * np.cos(X) * np.cos(Y) + 0.05 * np.cos(2 * X) * np.sin(Z)
    u = 0.2 * np.sin(X) * np.cos(Z) + 0.1 * np.sin(2 * X) * np.sin(Y)
    v = 0.1 + 0.2 * np.cos(X) * np.sin(Z)
    w = -0.1 + 0.1 * np.cos(2 * X) * np.cos(Y)
    p = 1.0 + 0.1 * np.cos(X) * np.sin(Y) * np.cos(Z)
    return wl.prim_to_cons_np(rho, u, v, w, p, 1.4)


@pytest.mark.parametrize("riemann", [ROE, HLLC, RUSANOV])
@pytest.mark.parametrize("nt", [0, 1])
def test_slip_wall_equals_mirrored_periodic_domain(riemann, nt):
    """Inviscid: a slip wall sees the mirror image of the inner state, exactly what
    the symmetry plane of a mirror-symmetric periodic flow sees; the right-hand side
    on [0, pi] x [0, 2 pi]^2 with slip walls at x = 0, pi equals that of the
    periodic [-pi, pi] x [0, 2 pi]^2 flow on its x >= 0 half."""
    N = 3
    A = wl.box_mesh((2, 2, 2), lo=(0.0, 0.0, 0.0), hi=(math.pi, 2 * math.pi, 2 * math.pi),
                    periodic=(False, True, True), bc_ids=[1, 1, 0, 0, 0, 0])
    B = wl.box_mesh((4, 2, 2), lo=(-math.pi, 0.0, 0.0), hi=(math.pi, 2 * math.pi, 2 * math.pi))
    pa = Params(N=N, node_type=nt, riemann=riemann, mu=0.0, bc_kinds={1: BC_SLIP_WALL})
    pb = Params(N=N, node_type=nt, riemann=riemann, mu=0.0)
    Ra = DGSEM(pa, A.coords, A.conn).rhs(T(_mirror_state(A.node_coords(N, nt))))
    Rb = DGSEM(pb, B.coords, B.conn).rhs(T(_mirror_state(B.node_coords(N, nt))))
    # element (a, b, c) of A is element (a + 2, b, c) of B (identity frames, x-fastest lattice)
    idx = [int(np.nonzero((B.lattice == A.lattice[e] + np.array([2, 0, 0])).all(1))[0][0]) for e in range(A.K)]
    d = (Ra - Rb[idx]).abs().max() / Rb.abs().max()
    assert float(d) < 1e-12


@pytest.mark.parametrize("riemann", [ROE, HLLC])
@pytest.mark.parametrize("mu", [0.0, 1.0 / 400.0])
def test_closed_box_slip_walls_conserve(riemann, mu):
    """Curved box closed by slip walls on all six sides: the mirror state makes the
    wall's mass flux vanish, so total mass is conserved to round-off; for mu = 0
    the energy flux vanishes too."""
    N = 3
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3,
                    reorient_seed=3, bc_ids=[2] * 6)
    dg = DGSEM(Params(N=N, riemann=riemann, mu=mu, bc_kinds={2: BC_SLIP_WALL}), m.coords, m.conn)
    Ut = dg.rhs(T(wl.perturbed(np.pi * m.node_coords(N, 0), seed=6)))
    wJ = dg.quad_weights().unsqueeze(1)
    tot = (wJ * Ut).sum(dim=(0, 2, 3, 4))
    scale = (wJ * Ut.abs()).sum(dim=(0, 2, 3, 4))
    assert float(abs(tot[0]) / scale[0]) < 1e-13
    if mu == 0.0:
        assert float(abs(tot[4]) / scale[4]) < 1e-13
    else:
        assert float(abs(tot[4]) / scale[4]) > 1e-10  # the wall's viscous stress does work


@pytest.mark.parametrize("nt", [0, 1])
def test_slip_walls_keep_a_fluid_at_rest(nt):
    N = 4
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3,
                    reorient_seed=5, bc_ids=[2] * 6)
    dg = DGSEM(Params(N=N, node_type=nt, riemann=HLLC, bc_kinds={2: BC_SLIP_WALL}), m.coords, m.conn)
    U = T(wl.freestream(m.node_coords(N, nt), vel=(0.0, 0.0, 0.0)))
    assert float(dg.rhs(U).abs().max()) < 1e-12


@pytest.mark.parametrize("nt", [0, 1])
def test_exact_inflow_outflow_freestream(nt):
    """Free stream entering through exact-state sides (x = -1) and leaving through
    outflow sides (x = +1) of a curved mesh: the right-hand side vanishes."""
    N = 4
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False, True, True),
                    reorient_seed=2, bc_ids=[0, 1, 0, 0, 0, 0])
    dg = DGSEM(Params(N=N, node_type=nt, riemann=ROE, bc_exact=eq.EXACT_FREESTREAM, bc_kinds={1: BC_OUTFLOW}),
               m.coords, m.conn)
    assert float(dg.rhs(T(wl.freestream(m.node_coords(N, nt)))).abs().max()) < 1e-12


def test_outflow_side_sees_no_jump():
    """An outflow side's outer state is the inner one, so its numerical flux is the
    physical flux F(U_L).n: changing the exact-state function must not change U_t
    when every boundary is an outflow."""
    N = 2
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, periodic=(False,) * 3, bc_ids=[3] * 6)
    U = T(wl.perturbed(np.pi * m.node_coords(N, 0), seed=2))
    r = [DGSEM(Params(N=N, riemann=HLLC, bc_exact=k, bc_kinds={3: BC_OUTFLOW}), m.coords, m.conn).rhs(U)
         for k in (eq.EXACT_FREESTREAM, eq.EXACT_MANUFACTURED)]
    assert torch.equal(r[0], r[1])
    e = DGSEM(Params(N=N, riemann=HLLC, bc_exact=eq.EXACT_FREESTREAM, bc_kinds={3: BC_EXACT}), m.coords,
              m.conn).rhs(U)
    assert float((e - r[0]).abs().max()) > 1e-6
