"""Pins of the oracle's time integration (Sec. 3.4, Williamson low-storage RK with
the Carpenter-Kennedy 4(5) coefficients) and of its discrete adjoint."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import equations as eq
from oracle.dgsem import DGSEM, RK_A, RK_B, RK_C, ROE, Params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def butcher_from_2n(A, B):
    """Butcher tableau (a, b) of the 2N-storage scheme dU = A dU + h f; U += B dU."""
    s = len(A)
    a = np.zeros((s + 1, s))
    for k in range(1, s + 1):  # row k+1 uses stages 1..k
        for j in range(1, k + 1):
            tot = 0.0
            for m in range(j, k + 1):
                prod = 1.0
                for r in range(j + 1, m + 1):
                    prod *= A[r - 1]
                tot += B[m - 1] * prod
            a[k, j - 1] = tot
    return a[:s], a[s]


def test_coefficients_match_published():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "lserk45_carpenter_kennedy.txt")) if l.strip() and l[0] != "#"]
    for k, (stage, A, B, c) in enumerate(rows):
        assert float(Fraction(A)) == RK_A[k] and float(Fraction(B)) == RK_B[k] and float(Fraction(c)) == RK_C[k]


def test_lserk_order_conditions():
    a, b = butcher_from_2n(RK_A, RK_B)
    c = a.sum(1)
    assert np.allclose(c, RK_C, atol=1e-12, rtol=0)
    conds = [(b.sum(), 1.0), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ (a @ c), 1 / 6), (b @ c ** 3, 1 / 4),
             (b @ (c * (a @ c)), 1 / 8), (b @ (a @ c ** 2), 1 / 12), (b @ (a @ (a @ c)), 1 / 24)]
    for val, exact in conds:
        assert abs(val - exact) < 1e-12
    # not 5th order: one fifth-order condition fails clearly
    assert abs(b @ c ** 4 - 1 / 5) > 1e-6


def _rk_scalar(f, y0, h, nsteps):
    y, dy, t = y0, 0.0, 0.0
    for _ in range(nsteps):
        for k in range(5):
            dy = RK_A[k] * dy + h * f(t + RK_C[k] * h, y)
            y = y + RK_B[k] * dy
        t += h
    return y


def test_linear_stability_polynomial():
    """One step on y' = lam y gives the degree-5 stability polynomial whose first
    five Taylor coefficients are 1/k! (fourth order)."""
    a, b = butcher_from_2n(RK_A, RK_B)
    for z in (0.1, -0.7, -2.3):
        y1 = _rk_scalar(lambda t, y: z * y, 1.0, 1.0, 1)
        # R(z) = 1 + z b^T (I - z a)^{-1} 1
        R = 1 + z * b @ np.linalg.solve(np.eye(5) - z * a, np.ones(5))
        assert abs(y1 - R) < 1e-14 * max(1, abs(R))
        assert abs(R - sum(z ** k / math.factorial(k) for k in range(5))) < abs(z) ** 5 * 0.05


def test_observed_fourth_order():
    f = lambda t, y: -y * y + math.cos(t)  # nonlinear, non-autonomous
    ref = _rk_scalar(f, 1.0, 1e-3, 2000)
    errs = [abs(_rk_scalar(f, 1.0, 2.0 / n, n) - ref) for n in (20, 40, 80)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 3.8


# ---------------------------------------------------------------------- adjoint
def _small_tgv(N=2, nelem=(2, 2, 2)):
    m = wl.box_mesh(nelem, Ngeo=1, reorient_seed=3)
    dg = DGSEM(Params(N=N, node_type=0, riemann=ROE, smooth_roe=True, mu=1.0 / 400.0), m.coords, m.conn)
    x = m.node_coords(N, 0)
    U0 = torch.tensor(wl.taylor_green(x) + 0.01 * (wl.perturbed(x, seed=2) - wl.perturbed(x, seed=2).mean()))
    return m, dg, U0


def test_adjoint_matches_central_fd():
    """dJ/dU0 of J = KE(U_T) by the discrete adjoint vs central finite differences
    (eps = 1e-6) in seeded random directions."""
    m, dg, U0 = _small_tgv()
    dt, nsteps = 1e-3, 3
    Jv, grad = dg.gradient_ke(U0, nsteps, dt)
    for v in wl.random_directions(U0.shape, 3, seed0=1910):
        v = torch.tensor(v)
        eps = 1e-6
        Jp = float(dg.kinetic_energy(dg.run(U0 + eps * v, nsteps, dt)))
        Jm = float(dg.kinetic_energy(dg.run(U0 - eps * v, nsteps, dt)))
        fd = (Jp - Jm) / (2 * eps)
        ad = float((grad * v).sum())
        assert abs(fd - ad) < 1e-6 * max(abs(ad), 1e-3), (fd, ad)


def test_adjoint_dot_product_forward_mode():
    """<lam, (dL/dU) v> (forward mode) = <(dL/dU)^T lam, v> (reverse mode)."""
    from torch.func import jvp

    m, dg, U0 = _small_tgv()
    rng = np.random.default_rng(4)
    v = torch.tensor(rng.normal(size=U0.shape))
    lam = torch.tensor(rng.normal(size=U0.shape))
    _, Jv = jvp(lambda U: dg.rhs(U), (U0,), (v,))
    JTl = dg.rhs_vjp(U0, 0.0, lam)
    a, b = float((lam * Jv).sum()), float((JTl * v).sum())
    assert abs(a - b) < 1e-12 * max(abs(a), 1.0)


@pytest.mark.parametrize("kinds", [{1: 1, 2: 2}, {1: 0, 2: 1}])
def test_adjoint_with_boundaries_matches_central_fd(kinds):
    """Curved box with exact-state, outflow and slip-wall sides and the
    manufactured source at t = 0.3: <lam, (L(U + eps v) - L(U - eps v)) / (2 eps)>
    equals <(dL/dU)^T lam, v> (the outer boundary states depend on the inner
    ones; the exact state and the source do not).  Kinds: 0 exact state,
    1 outflow, 2 slip wall; bc_id 0 is always an exact-state side."""
    N = 2
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=2, mapping="sine", periodic=(False,) * 3,
                    reorient_seed=3, bc_ids=[0, 1, 2, 2, 1, 2])
    dg = DGSEM(Params(N=N, riemann=ROE, smooth_roe=True, mu=1.0 / 400.0, bc_exact=2, source=True,
                      bc_kinds=dict(kinds)), m.coords, m.conn)
    x = m.node_coords(N, 0)
    U0 = torch.tensor(wl.perturbed(np.pi * x, seed=3))
    rng = np.random.default_rng(5)
    v = torch.tensor(rng.normal(size=U0.shape))
    lam = torch.tensor(rng.normal(size=U0.shape))
    eps = 1e-6
    Jv = (dg.rhs(U0 + eps * v, 0.3) - dg.rhs(U0 - eps * v, 0.3)) / (2 * eps)
    a, b = float((lam * Jv).sum()), float((dg.rhs_vjp(U0, 0.3, lam) * v).sum())
    assert abs(a - b) < 1e-7 * abs(b), (a, b)


@pytest.mark.parametrize("variant", ["kep", "ec", "br2", "mortar"])
def test_adjoint_of_other_forms_matches_central_fd(variant):
    """The oracle's reverse mode for the split forms (LGL), BR2 and a mortar mesh
    against a central difference of its own RHS in a random direction."""
    from oracle.dgsem import EC

    N = 2
    rng = np.random.default_rng(12)
    if variant == "mortar":
        m = wl.mortar_box_mesh(refine=(1, 2, 2), ny=1, nz=1, reorient_seed=3)
        dg = DGSEM(Params(N=N, riemann=ROE, smooth_roe=True, mu=1.0 / 400.0), m.coords, m.conn, m.mortars)
        nt = 0
    else:
        m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=2, mapping="sine", periodic=(False,) * 3,
                        reorient_seed=2, bc_ids=[0, 1, 2, 2, 1, 0])
        kw = dict(bc_kinds={1: 1, 2: 2})
        # smooth surface fluxes (smoothed Roe, EC): a central difference across a kink of
        # HLLC's wave-speed or star-region switches would not measure the derivative
        if variant == "br2":
            kw.update(lifting="br2", eta_br2=3.0)
            nt, riem = 0, ROE
        else:
            kw.update(split="pirozzoli" if variant == "kep" else "chandrashekar")
            nt, riem = 1, (ROE if variant == "kep" else EC)
        dg = DGSEM(Params(N=N, node_type=nt, riemann=riem, smooth_roe=riem == ROE, mu=1.0 / 400.0, bc_exact=1, **kw),
                   m.coords, m.conn)
    U0 = torch.tensor(wl.perturbed(np.pi * m.node_coords(N, nt), seed=5))
    v = torch.tensor(rng.normal(size=U0.shape))
    lam = torch.tensor(rng.normal(size=U0.shape))
    eps = 1e-6
    Jv = (dg.rhs(U0 + eps * v, 0.2) - dg.rhs(U0 - eps * v, 0.2)) / (2 * eps)
    a, b = float((lam * Jv).sum()), float((dg.rhs_vjp(U0, 0.2, lam) * v).sum())
    assert abs(a - b) < 1e-7 * abs(b), (a, b)
