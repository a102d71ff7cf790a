"""Pins of the entropy-conservative split form (Sec. 3.3: split forms that mimic
the continuous kinetic-energy or entropy balance; Chandrashekar's two-point flux
with logarithmic means) and of its entropy-conservative surface flux."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import equations as eq
from oracle.dgsem import DGSEM, EC, HLLC, ROE, Params

GAMMA = 1.4
GAS = eq.Gas(GAMMA, 0.72, 0.0)


def T(a):
    return torch.tensor(a, dtype=torch.float64)


def test_log_mean():
    """Against the definition evaluated in 40-digit arithmetic (mpmath), for well
    separated and for nearly equal arguments (where the quotient form loses digits)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(1)
    a = 0.5 + rng.random(60)
    b = np.concatenate([0.5 + rng.random(20), a[20:40] * (1 + 1e-3 * rng.normal(size=20)),
                        a[40:] * (1 + 1e-9 * rng.normal(size=20))])
    exact = [float((mpmath.mpf(x) - mpmath.mpf(y)) / (mpmath.log(x) - mpmath.log(y))) if x != y else x
             for x, y in zip(a, b)]
    assert torch.allclose(eq.log_mean(T(a), T(b)), T(exact), rtol=4e-15, atol=0)
    a, b = T(a), T(b)
    assert torch.allclose(eq.log_mean(a, b), eq.log_mean(b, a), rtol=1e-15, atol=0)
    assert torch.allclose(eq.log_mean(a, a), a, rtol=1e-15, atol=0)
    # close arguments: between the geometric and the arithmetic mean (both tend to it)
    c = a * (1 + 1e-7)
    lm = eq.log_mean(a, c)
    assert bool(((lm >= torch.sqrt(a * c) * (1 - 1e-15)) & (lm <= 0.5 * (a + c) * (1 + 1e-15))).all())


def test_chandrashekar_flux_consistent_and_symmetric():
    rng = np.random.default_rng(3)

    def state():
        W = T(np.column_stack([0.8 + rng.random(40), rng.normal(size=(40, 3)), 0.8 + rng.random(40)]))
        return eq.cons(W, GAS), W

    (Ua, Wa), (Ub, Wb) = state(), state()
    Ja, Jb = T(rng.normal(size=(40, 3))), T(rng.normal(size=(40, 3)))
    f = eq.two_point_contravariant(Ua, Wa, Ua, Wa, Ja, Ja, "chandrashekar", GAMMA)
    ref = (eq.flux_conv(Ua, Wa) * Ja.unsqueeze(-1)).sum(-2)
    assert torch.allclose(f, ref, rtol=1e-13, atol=1e-13)
    fab = eq.two_point_contravariant(Ua, Wa, Ub, Wb, Ja, Jb, "chandrashekar", GAMMA)
    fba = eq.two_point_contravariant(Ub, Wb, Ua, Wa, Jb, Ja, "chandrashekar", GAMMA)
    assert torch.allclose(fab, fba, rtol=1e-14, atol=1e-14)


def _entropy_variables(U):
    """v = dS/dU for S = -rho s / (gamma - 1), s = ln(p rho^-gamma)."""
    W = eq.prim(U.movedim(1, -1), GAS)
    rho, u, p = W[..., 0], W[..., 1:4], W[..., 4]
    s = torch.log(p) - GAMMA * torch.log(rho)
    beta = rho / p
    v1 = (GAMMA - s) / (GAMMA - 1.0) - 0.5 * beta * (u * u).sum(-1)
    return torch.cat([v1.unsqueeze(-1), beta.unsqueeze(-1) * u, -beta.unsqueeze(-1)], -1).movedim(-1, 1)


def _rough_state(x, seed):
    rng = np.random.default_rng(seed)
    sh = x[:, 0].shape
    return wl.prim_to_cons_np(1 + 0.2 * rng.random(sh), 0.3 * rng.normal(size=sh), 0.3 * rng.normal(size=sh),
                              0.3 * rng.normal(size=sh), 1 + 0.2 * rng.random(sh), GAMMA)


def _entropy_rate(N, mapping, riemann, split, seed=0):
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N if mapping == "sine" else 1, mapping=mapping,
                    reorient_seed=3)
    U = T(_rough_state(m.node_coords(N, 1), seed))
    dg = DGSEM(Params(N=N, node_type=1, riemann=riemann, mu=0.0, split=split), m.coords, m.conn)
    vUt = dg.quad_weights().unsqueeze(1) * _entropy_variables(U) * dg.rhs(U)
    return float(vUt.sum()), float(vUt.abs().sum())


@pytest.mark.parametrize("N,mapping", [(2, "cartesian"), (3, "cartesian"), (4, "sine"), (5, "sine")])
def test_entropy_conserved_with_ec_volume_and_surface_fluxes(N, mapping):
    """Inviscid, periodic, rough state: the EC split form with the EC surface flux
    conserves the discrete entropy sum_nodes wJ v . U_t to round-off, also on a
    curved mesh (metric averaging); the KEP volume flux does not."""
    rate, scale = _entropy_rate(N, mapping, EC, "chandrashekar")
    assert abs(rate) < 1e-11 * scale, (rate, scale)
    rate_kep, scale_kep = _entropy_rate(N, mapping, EC, "pirozzoli")
    assert abs(rate_kep) > 1e-6 * scale_kep


@pytest.mark.parametrize("riemann", [ROE, HLLC])
def test_dissipative_surface_fluxes_decrease_entropy(riemann):
    rate, scale = _entropy_rate(3, "sine", riemann, "chandrashekar")
    assert rate < -1e-3 * scale, (rate, scale)


def test_ec_split_freestream_and_conservation():
    N = 4
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3,
                    reorient_seed=2)
    dg = DGSEM(Params(N=N, node_type=1, riemann=EC, split="chandrashekar", bc_exact=eq.EXACT_FREESTREAM),
               m.coords, m.conn)
    assert float(dg.rhs(T(wl.freestream(m.node_coords(N, 1)))).abs().max()) < 1e-12
    mp = wl.box_mesh((3, 2, 2), Ngeo=1, reorient_seed=5)
    dgp = DGSEM(Params(N=3, node_type=1, riemann=HLLC, split="chandrashekar"), mp.coords, mp.conn)
    Ut = dgp.rhs(T(wl.perturbed(mp.node_coords(3, 1), seed=4)))
    wJ = dgp.quad_weights().unsqueeze(1)
    tot, sc = (wJ * Ut).sum(dim=(0, 2, 3, 4)), (wJ * Ut.abs()).sum(dim=(0, 2, 3, 4))
    assert float((tot.abs() / sc).max()) < 1e-13
