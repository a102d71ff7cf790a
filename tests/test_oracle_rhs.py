"""Pins of the oracle's right-hand side (Eq. semiDiscrete with BR1 lifting,
Eq. discreteGradient) against properties the paper and the mathematics fix:
free-stream preservation, discrete conservation, exact lifting of polynomials,
invariance under element reorientation, pointwise flux closed forms and the
initial Taylor-Green dissipation rate."""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import equations as eq
from oracle.dgsem import DGSEM, HLLC, ROE, RUSANOV, Params

GAS = eq.Gas(1.4, 0.72, 1.0 / 1600.0)


def T(a):
    return torch.tensor(a, dtype=torch.float64)


# ---------------------------------------------------------------- pointwise physics
def test_prim_cons_roundtrip():
    rng = np.random.default_rng(0)
    W = T(np.column_stack([1 + rng.random(20), rng.normal(size=(20, 3)), 1 + rng.random(20)]))
    assert torch.allclose(eq.prim(eq.cons(W, GAS), GAS), W, rtol=1e-14, atol=1e-14)


def test_convective_flux_closed_form():
    W = T([[1.3, 0.2, -0.4, 0.7, 2.1]])
    U = eq.cons(W, GAS)
    F = eq.flux_conv(U, W)[0]
    rho, u, v, w, p = W[0].tolist()
    E = p / 0.4 + 0.5 * rho * (u * u + v * v + w * w)
    vel = [u, v, w]
    for d in range(3):
        expect = [rho * vel[d]] + [rho * vel[c] * vel[d] + (p if c == d else 0) for c in range(3)] + [vel[d] * (E + p)]
        assert torch.allclose(F[d], T(expect), rtol=1e-14)


def test_viscous_flux_closed_forms():
    mu, g, Pr = GAS.mu, GAS.gamma, GAS.Pr
    W = T([[1.2, 0.3, -0.1, 0.2, 0.9]])
    # simple shear u = a*y: tau_xy = mu a
    G = torch.zeros(1, 3, 5, dtype=torch.float64)
    G[0, 1, 1] = 2.0
    Fv = eq.flux_visc(W, G, GAS)[0]
    assert torch.allclose(Fv[1], T([0, mu * 2, 0, 0, 0.3 * mu * 2]), rtol=1e-14)  # F^v_y
    assert torch.allclose(Fv[0], T([0, 0, mu * 2, 0, -0.1 * mu * 2]), rtol=1e-14)  # F^v_x: tau_yx
    # uniaxial compression u = a*x: tau_xx = 4/3 mu a, tau_yy = tau_zz = -2/3 mu a
    G = torch.zeros(1, 3, 5, dtype=torch.float64)
    G[0, 0, 1] = 1.5
    Fv = eq.flux_visc(W, G, GAS)[0]
    assert torch.allclose(Fv[0, 1], T(4 / 3 * mu * 1.5)) and torch.allclose(Fv[1, 2], T(-2 / 3 * mu * 1.5))
    # heat flux: T ~ p/rho linear in z via p only
    G = torch.zeros(1, 3, 5, dtype=torch.float64)
    G[0, 2, 4] = 0.6
    Fv = eq.flux_visc(W, G, GAS)[0]
    assert torch.allclose(Fv[2, 4], T(mu * g / ((g - 1) * Pr) * 0.6 / 1.2), rtol=1e-14)


def _rand_states(n, seed, Ma=0.5):
    rng = np.random.default_rng(seed)
    rho = 0.5 + rng.random(n)
    vel = rng.normal(size=(n, 3)) * Ma
    p = 0.5 + rng.random(n)
    return eq.cons(T(np.column_stack([rho, vel, p])), GAS)


def _rand_normals(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return T(v / np.linalg.norm(v, axis=1, keepdims=True))


@pytest.mark.parametrize("kind", ["roe", "roe_smooth", "hllc", "rusanov"])
def test_riemann_consistency_and_symmetry(kind):
    f = {"roe": lambda a, b, n: eq.riemann_roe(a, b, n, GAS),
         "roe_smooth": lambda a, b, n: eq.riemann_roe(a, b, n, GAS, smooth=True),
         "hllc": lambda a, b, n: eq.riemann_hllc(a, b, n, GAS),
         "rusanov": lambda a, b, n: eq.riemann_rusanov(a, b, n, GAS)}[kind]
    UL, UR, n = _rand_states(50, 1), _rand_states(50, 2), _rand_normals(50, 3)
    F = eq.normal_flux(eq.flux_conv(UL, eq.prim(UL, GAS)), n)
    assert torch.allclose(f(UL, UL, n), F, rtol=1e-13, atol=1e-13)
    assert torch.allclose(f(UL, UR, n), -f(UR, UL, -n), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind", ["roe", "hllc"])
def test_riemann_supersonic_upwinding(kind):
    """All waves to the right -> f* = F(U_L); all to the left -> F(U_R) (Roe
    property of the decomposition; HLLC wave structure)."""
    f = (lambda a, b, n: eq.riemann_roe(a, b, n, GAS)) if kind == "roe" else (lambda a, b, n: eq.riemann_hllc(a, b, n, GAS))
    n = T([[0.0, 0.6, 0.8]])
    WL = T([[1.0, 0.1, 3.0 * 0.6, 3.0 * 0.8, 0.7]])
    WR = T([[1.2, -0.2, 3.2 * 0.6, 3.2 * 0.8, 0.8]])
    UL, UR = eq.cons(WL, GAS), eq.cons(WR, GAS)
    FL = eq.normal_flux(eq.flux_conv(UL, WL), n)
    assert torch.allclose(f(UL, UR, n), FL, rtol=1e-13, atol=1e-13)
    WL2 = T([[1.0, 0.1, -3.0 * 0.6, -3.0 * 0.8, 0.7]])
    WR2 = T([[1.2, -0.2, -3.2 * 0.6, -3.2 * 0.8, 0.8]])
    UL2, UR2 = eq.cons(WL2, GAS), eq.cons(WR2, GAS)
    FR2 = eq.normal_flux(eq.flux_conv(UR2, WR2), n)
    assert torch.allclose(f(UL2, UR2, n), FR2, rtol=1e-13, atol=1e-13)


def test_rusanov_closed_form():
    """Scalar-dissipation flux: the jump is damped by the largest local wave speed."""
    n = T([[1.0, 0.0, 0.0]])
    WL, WR = T([[1.0, 0.5, 0.0, 0.0, 1.0]]), T([[1.0, 0.5, 0.0, 0.0, 2.0]])
    UL, UR = eq.cons(WL, GAS), eq.cons(WR, GAS)
    lam = max(0.5 + math.sqrt(1.4 * 1.0), 0.5 + math.sqrt(1.4 * 2.0))
    FL = eq.normal_flux(eq.flux_conv(UL, WL), n)
    FR = eq.normal_flux(eq.flux_conv(UR, WR), n)
    assert torch.allclose(eq.riemann_rusanov(UL, UR, n, GAS), 0.5 * (FL + FR) - 0.5 * lam * (UR - UL), rtol=1e-15)


def test_hllc_resolves_stationary_contact():
    n = T([[1.0, 0.0, 0.0]])
    WL, WR = T([[1.0, 0.0, 0.3, 0.0, 1.0]]), T([[0.2, 0.0, -0.5, 0.1, 1.0]])
    f = eq.riemann_hllc(eq.cons(WL, GAS), eq.cons(WR, GAS), n, GAS)
    assert torch.allclose(f, T([[0.0, 1.0, 0.0, 0.0, 0.0]]), atol=1e-14)


# ---------------------------------------------------------------- assembled operator
def _dg(nelem, N, nt, riemann=ROE, mapping="cartesian", periodic=True, reo=None, Ngeo=1, lo=(0.0,) * 3,
        hi=(2 * math.pi,) * 3, **kw):
    per = (periodic,) * 3 if isinstance(periodic, bool) else periodic
    m = wl.box_mesh(nelem, lo=lo, hi=hi, Ngeo=Ngeo, periodic=per, mapping=mapping, reorient_seed=reo)
    return m, DGSEM(Params(N=N, node_type=nt, riemann=riemann, **kw), m.coords, m.conn)


@pytest.mark.parametrize("nt", [0, 1])
@pytest.mark.parametrize("riemann", [ROE, HLLC, RUSANOV])
def test_freestream_curved(nt, riemann):
    """Free-stream preservation on a curved mesh (Sec. 3.1, curl metrics)."""
    N = 4
    m, dg = _dg((3, 2, 2), N, nt, riemann, mapping="sine", periodic=False, reo=4, Ngeo=N, lo=(-1,) * 3, hi=(1,) * 3,
                bc_exact=eq.EXACT_FREESTREAM)
    U = T(wl.freestream(m.node_coords(N, nt)))
    Ut = dg.rhs(U)
    assert Ut.abs().max() < 5e-12


@pytest.mark.parametrize("nt", [0, 1])
@pytest.mark.parametrize("riemann", [ROE, HLLC, RUSANOV])
@pytest.mark.parametrize("state", ["tgv", "perturbed"])
def test_conservation_periodic(nt, riemann, state):
    """sum_nodes w J U_t = 0 for all five conserved variables (the side flux is
    single-valued, added with opposite signs on the two elements)."""
    N = 3
    m, dg = _dg((3, 3, 2), N, nt, riemann, reo=2)
    x = m.node_coords(N, nt)
    U = T(wl.taylor_green(x) if state == "tgv" else wl.perturbed(x, seed=5))
    Ut = dg.rhs(U)
    tot = (dg.quad_weights().unsqueeze(1) * Ut).sum(dim=(0, 2, 3, 4))
    scale = (dg.quad_weights().unsqueeze(1) * Ut.abs()).sum(dim=(0, 2, 3, 4))
    assert (tot.abs() / scale).max() < 1e-13


def _local_to_identity_perm(m, N):
    """For a reoriented BoxMesh: index map so that field_reo[e].flatten()[perm[e]]
    is in identity-frame node order."""
    n = N + 1
    perm = np.zeros((m.K, n ** 3), dtype=np.int64)
    idx = np.arange(n)
    for e in range(m.K):
        R = m.frames[e]
        for kk in range(n):
            for jj in range(n):
                for ii in range(n):
                    loc = np.array([ii, jj, kk])
                    # eta = R xi with xi_a = r[loc_a] -> identity-frame index along axis g
                    gidx = np.zeros(3, dtype=np.int64)
                    for g in range(3):
                        a = int(np.nonzero(R[g])[0][0])
                        gidx[g] = loc[a] if R[g, a] > 0 else N - loc[a]
                    perm[e, gidx[2] * n * n + gidx[1] * n + gidx[0]] = kk * n * n + jj * n + ii
    return perm


@pytest.mark.parametrize("nt", [0, 1])
def test_reorientation_invariance(nt):
    """Element local frames and side flips must not change the result (Sec. 5.1)."""
    N = 3
    m0, dg0 = _dg((3, 2, 2), N, nt, HLLC)
    m1, dg1 = _dg((3, 2, 2), N, nt, HLLC, reo=9)
    U0 = T(wl.perturbed(m0.node_coords(N, nt), seed=3))
    U1 = T(wl.perturbed(m1.node_coords(N, nt), seed=3))
    R0, R1 = dg0.rhs(U0), dg1.rhs(U1)
    perm = torch.tensor(_local_to_identity_perm(m1, N))
    R1i = torch.gather(R1.flatten(2), 2, perm.unsqueeze(1).expand(-1, 5, -1)).view_as(R0)
    assert (R0 - R1i).abs().max() < 1e-12 * R0.abs().max()


@pytest.mark.parametrize("nt", [0, 1])
def test_lifting_exact_for_polynomials(nt):
    """BR1 lifting (Eq. discreteGradient) returns the exact gradient of a
    continuous polynomial field of degree <= N, with exact Dirichlet data.  LGL:
    all primitives; LG: rho and p with zero velocity (the face state is W(U_face))."""
    N = 3
    rng = np.random.default_rng(1)
    C = rng.normal(size=(5, 4)) * 0.1  # linear-to-cubic coefficients per variable

    def W_of(x):  # x [..., 3]
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        ws = []
        for v in range(5):
            base = [1.0, 0.3, 0.2, 0.1, 1.0][v]
            f = base + C[v, 0] * X + C[v, 1] * Y * Z + C[v, 2] * X * X * Y + C[v, 3] * Z ** 3
            if nt == 0 and v in (1, 2, 3):
                f = torch.zeros_like(X)
            ws.append(f)
        return torch.stack(ws, -1)

    def gradW(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        out = torch.zeros(*x.shape[:-1], 3, 5, dtype=x.dtype)
        for v in range(5):
            if nt == 0 and v in (1, 2, 3):
                continue
            out[..., 0, v] = C[v, 0] + 2 * C[v, 2] * X * Y
            out[..., 1, v] = C[v, 1] * Z + C[v, 2] * X * X
            out[..., 2, v] = C[v, 1] * Y + 3 * C[v, 3] * Z * Z
        return out

    m, dg = _dg((2, 2, 2), N, nt, ROE, periodic=False, lo=(-1,) * 3, hi=(1,) * 3,
                bc_exact=lambda x, t: eq.cons(W_of(x), GAS))
    x = dg.geo.x.movedim(1, -1)
    U = eq.cons(W_of(x), GAS).movedim(-1, 1)
    _, parts = dg.rhs(U, parts=True)
    G = parts["G"].permute(0, 3, 4, 5, 1, 2)  # [K,n,n,n,3,5]
    assert (G - gradW(x)).abs().max() < 1e-12


def test_tgv_initial_dissipation_rate():
    """dKE/dt at t=0 for the Taylor-Green vortex equals -mu <|omega|^2> V =
    -mu (3/4)(2 pi)^3 in the incompressible limit (closed form for the initial
    field); the DG value at N=5, 4^3 must agree to within the O(Ma^2) and
    discretisation error."""
    N = 5
    m, dg = _dg((4, 4, 4), N, 0, ROE, Ma=0.1)
    U = T(wl.taylor_green(m.node_coords(N, 0)))
    Ut = dg.rhs(U)
    with torch.enable_grad():
        Ux = U.clone().requires_grad_(True)
        (dke,) = torch.autograd.grad(dg.kinetic_energy(Ux), Ux)
    rate = float((dke * Ut).sum())
    exact = -GAS.mu * 0.75 * (2 * math.pi) ** 3
    assert abs(rate - exact) < 0.03 * abs(exact)
    # a wrong viscous operator (mu scaled) would miss by far more
    ke = float(dg.kinetic_energy(U))
    assert abs(ke - 0.125 * (2 * math.pi) ** 3) < 1e-3 * ke
