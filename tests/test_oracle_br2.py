"""Pins of the oracle's BR2 face gradients (Bassi & Rebay 1997, named by the paper
beside BR1): on each side of a face the viscous flux takes the broken gradient
plus eta times that face's own lifting; the volume integral keeps the BR1 gradient."""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import equations as eq
from oracle.dgsem import DGSEM, HLLC, ROE, Params

GAS = eq.Gas(1.4, 0.72, 1.0 / 1600.0)


def T(a):
    return torch.tensor(a, dtype=torch.float64)


def _piecewise(m, N, nt, moving):
    """Per element its own quadratic primitive field (discontinuous across elements)
    and the exact gradient; zero velocity when not moving (the face primitives are
    W(U_face), linear in U only without velocity)."""
    x = T(m.node_coords(N, nt))
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    rng = np.random.default_rng(0)
    C = T(rng.normal(size=(m.K, 5, 3)))
    c = lambda v, q: C[:, v, q].view(-1, 1, 1, 1)
    base = [1.0, 0.2, -0.1, 0.1, 1.0]
    on = [1.0, float(moving), float(moving), float(moving), 1.0]
    W = torch.stack([base[v] * on[v] + on[v] * 0.05 * (c(v, 0) * X + c(v, 1) * Y * Z + c(v, 2) * X * X)
                     for v in range(5)], 1)
    dW = torch.stack([torch.stack([on[v] * 0.05 * (c(v, 0) + 2 * c(v, 2) * X) for v in range(5)], 1),
                      torch.stack([on[v] * 0.05 * c(v, 1) * Z for v in range(5)], 1),
                      torch.stack([on[v] * 0.05 * c(v, 1) * Y for v in range(5)], 1)], 1)
    return eq.cons(W.movedim(1, -1), GAS).movedim(-1, 1), dW


@pytest.mark.parametrize("nt,moving", [(1, True), (0, False)])
def test_br2_without_penalty_gives_the_broken_gradient(nt, moving):
    """eta = 0: the BR2 face gradient is the trace of each element's own gradient,
    exactly for a piecewise polynomial field on affine elements, although the field
    jumps across every face."""
    N = 3
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, reorient_seed=4)
    U, dW = _piecewise(m, N, nt, moving)
    dg = DGSEM(Params(N=N, node_type=nt, riemann=HLLC, lifting="br2", eta_br2=0.0), m.coords, m.conn)
    _, parts = dg.rhs(U, parts=True)
    ref = dg.geo.face_values(dW.flatten(1, 2), dg.b.l_side)
    RL, RR = dg.geo.master_slave(ref)
    assert float((parts["GL"] - RL).abs().max()) < 1e-12 * float(RL.abs().max())
    assert float((parts["GR"] - RR).abs().max()) < 1e-12 * float(RL.abs().max())


def test_br2_equals_br1_for_continuous_polynomials():
    """No jumps (a global polynomial of degree <= N): every lifting vanishes and BR2
    gives the BR1 right-hand side."""
    N = 3
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=1, periodic=(False,) * 3, reorient_seed=2)
    x = T(m.node_coords(N, 1))
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    W = torch.stack([1 + 0.1 * X * Y, 0.2 + 0.1 * Z, 0.1 * X * X, -0.1 + 0.05 * Y, 1 + 0.1 * X * Z], 1)
    U = eq.cons(W.movedim(1, -1), GAS).movedim(-1, 1)
    exact = lambda xb, t: eq.cons(torch.stack([1 + 0.1 * xb[..., 0] * xb[..., 1], 0.2 + 0.1 * xb[..., 2],
                                               0.1 * xb[..., 0] ** 2, -0.1 + 0.05 * xb[..., 1],
                                               1 + 0.1 * xb[..., 0] * xb[..., 2]], -1), GAS)
    r = [DGSEM(Params(N=N, node_type=1, riemann=HLLC, lifting=lift, bc_exact=exact), m.coords, m.conn).rhs(U)
         for lift in ("br1", "br2")]
    assert float((r[0] - r[1]).abs().max()) < 1e-12 * float(r[0].abs().max())


def test_br2_differs_from_br1_and_conserves():
    N = 3
    m = wl.box_mesh((3, 2, 2), reorient_seed=5)
    U = T(wl.perturbed(m.node_coords(N, 0), seed=9))
    r1 = DGSEM(Params(N=N, riemann=ROE, mu=0.01), m.coords, m.conn).rhs(U)
    dg2 = DGSEM(Params(N=N, riemann=ROE, mu=0.01, lifting="br2"), m.coords, m.conn)
    r2 = dg2.rhs(U)
    assert float((r1 - r2).abs().max()) > 1e-8 * float(r1.abs().max())
    wJ = dg2.quad_weights().unsqueeze(1)
    tot, sc = (wJ * r2).sum(dim=(0, 2, 3, 4)), (wJ * r2.abs()).sum(dim=(0, 2, 3, 4))
    assert float((tot.abs() / sc).max()) < 1e-13


def test_br2_freestream_curved():
    N = 4
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3,
                    reorient_seed=1)
    dg = DGSEM(Params(N=N, riemann=HLLC, lifting="br2", bc_exact=eq.EXACT_FREESTREAM), m.coords, m.conn)
    assert float(dg.rhs(T(wl.freestream(m.node_coords(N, 0)))).abs().max()) < 1e-12


def _mms_error(N, nel, lifting):
    m = wl.box_mesh((nel,) * 3, lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3)
    mu = 0.02  # viscous terms large enough that the face gradients matter
    gas = eq.Gas(1.4, 0.72, mu)
    dg = DGSEM(Params(N=N, riemann=HLLC, mu=mu, bc_exact=eq.EXACT_MANUFACTURED, source=True, lifting=lifting),
               m.coords, m.conn)
    x = dg.geo.x.movedim(1, -1)
    U0 = eq.exact_state(eq.EXACT_MANUFACTURED, x, 0.0, gas).movedim(-1, 1).contiguous()
    t_end = 0.05
    nsteps = int(math.ceil(t_end / (0.1 / nel / (N + 1))))
    U = dg.run(U0, nsteps, t_end / nsteps)
    Ue = eq.exact_state(eq.EXACT_MANUFACTURED, x, t_end, gas).movedim(-1, 1)
    return math.sqrt(float((dg.quad_weights() * (U[:, 0] - Ue[:, 0]) ** 2).sum()))


def test_br2_manufactured_convergence():
    """Curved mesh, manufactured solution with mu = 0.02: BR2 converges like BR1
    (order > N at N = 2 between 4^3 and 8^3 elements)."""
    N = 2
    e2 = [_mms_error(N, nel, "br2") for nel in (2, 4, 8)]
    e1 = [_mms_error(N, nel, "br1") for nel in (2, 4, 8)]
    order = lambda e: math.log2(e[1] / e[2])
    assert e2[0] > e2[1] > e2[2] and order(e2) > N, (e2, order(e2))
    assert abs(order(e2) - order(e1)) < 0.5, (order(e2), order(e1))
