"""Pins of the oracle's split-form DG operator (Sec. 3.3, Eq. semiDiscreteSplit;
Pirozzoli's kinetic-energy-preserving flux of the paper's NACA computation)."""
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


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_central_split_equals_standard_dgsem(N):
    """With the central two-point flux (F(a) + F(b))/2 and constant metrics (Cartesian
    elements) the split volume term 2 sum_a D_ia F#(i, a) equals D F, and the strong
    form equals the weak form on LGL nodes (summation by parts): the split operator
    must reproduce the standard operator to round-off."""
    m = wl.box_mesh((3, 2, 2), Ngeo=1, reorient_seed=N)
    U = T(wl.perturbed(m.node_coords(N, 1), seed=2))
    std = DGSEM(Params(N=N, node_type=1, riemann=HLLC), m.coords, m.conn).rhs(U)
    cen = DGSEM(Params(N=N, node_type=1, riemann=HLLC, split="central"), m.coords, m.conn).rhs(U)
    assert float((cen - std).abs().max() / std.abs().max()) < 1e-12


def test_pirozzoli_flux_consistent_and_symmetric():
    rng = np.random.default_rng(3)
    W = T(np.column_stack([1 + rng.random(30), rng.normal(size=(30, 3)), 1 + rng.random(30)]))
    W2 = T(np.column_stack([1 + rng.random(30), rng.normal(size=(30, 3)), 1 + rng.random(30)]))
    U, U2 = eq.cons(W, GAS), eq.cons(W2, GAS)
    Ja, Ja2 = T(rng.normal(size=(30, 3))), T(rng.normal(size=(30, 3)))
    f = eq.two_point_contravariant(U, W, U, W, Ja, Ja, "pirozzoli")
    ref = (eq.flux_conv(U, W) * Ja.unsqueeze(-1)).sum(-2)
    assert torch.allclose(f, ref, rtol=1e-13, atol=1e-13)
    fab = eq.two_point_contravariant(U, W, U2, W2, Ja, Ja2, "pirozzoli")
    fba = eq.two_point_contravariant(U2, W2, U, W, Ja2, Ja, "pirozzoli")
    assert torch.allclose(fab, fba, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("N", [2, 4])
def test_split_freestream_curved(N):
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3,
                    reorient_seed=1)
    dg = DGSEM(Params(N=N, node_type=1, riemann=HLLC, split="pirozzoli", bc_exact=eq.EXACT_FREESTREAM), m.coords,
               m.conn)
    assert float(dg.rhs(T(wl.freestream(m.node_coords(N, 1)))).abs().max()) < 5e-12


@pytest.mark.parametrize("riemann", [ROE, HLLC])
def test_split_conservation_periodic(riemann):
    N = 3
    m = wl.box_mesh((3, 2, 2), Ngeo=1, reorient_seed=5)
    dg = DGSEM(Params(N=N, node_type=1, riemann=riemann, split="pirozzoli"), m.coords, m.conn)
    Ut = dg.rhs(T(wl.perturbed(m.node_coords(N, 1), seed=4)))
    wJ = dg.quad_weights().unsqueeze(1)
    tot = (wJ * Ut).sum(dim=(0, 2, 3, 4))
    scale = (wJ * Ut.abs()).sum(dim=(0, 2, 3, 4))
    assert float((tot.abs() / scale).max()) < 1e-13


def test_split_not_standard_on_curved():
    """On curved elements the metric-averaged split form is a different operator
    (the product rule is not exact discretely): it must not coincide."""
    N = 3
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3)
    U = T(wl.manufactured(m.node_coords(N, 1), 0.0))
    std = DGSEM(Params(N=N, node_type=1, riemann=HLLC, bc_exact=eq.EXACT_MANUFACTURED), m.coords, m.conn).rhs(U)
    cen = DGSEM(Params(N=N, node_type=1, riemann=HLLC, bc_exact=eq.EXACT_MANUFACTURED, split="central"), m.coords,
                m.conn).rhs(U)
    assert float((cen - std).abs().max() / std.abs().max()) > 1e-8


def _mms_error(N, nel):
    m = wl.box_mesh((nel,) * 3, lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3)
    dg = DGSEM(Params(N=N, node_type=1, riemann=HLLC, bc_exact=eq.EXACT_MANUFACTURED, source=True,
                      split="pirozzoli"), m.coords, m.conn)
    x = dg.geo.x.movedim(1, -1)
    U0 = eq.exact_state(eq.EXACT_MANUFACTURED, x, 0.0, GAS).movedim(-1, 1).contiguous()
    t_end = 0.05
    nsteps = int(math.ceil(t_end / (0.1 / nel / (N + 1))))
    U = dg.run(U0, nsteps, t_end / nsteps)
    Ue = eq.exact_state(eq.EXACT_MANUFACTURED, x, t_end, GAS).movedim(-1, 1)
    return math.sqrt(float((dg.quad_weights() * (U[:, 0] - Ue[:, 0]) ** 2).sum()))


def test_split_manufactured_convergence():
    """Split form on the curved manufactured-solution case (LGL, N = 3): errors fall
    with order > N between the finest pair of meshes."""
    errs = [_mms_error(3, nel) for nel in (2, 4, 8)]
    order = math.log2(errs[1] / errs[2])
    assert errs[0] > errs[1] > errs[2] and order > 3, (errs, order)
