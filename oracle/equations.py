"""Compressible Navier-Stokes pointwise physics (oracle; test infrastructure only).

The paper writes the system abstractly (Eq. 3DconsLaw: U_t + div(F^c(U) -
F^v(U, grad U)) = 0, Sec. 3.1) and names its Riemann solvers (Roe, HLL-type,
Sec. 2.2) without formulas.  Readings, all standard ideal-gas forms:

* p = (gamma-1)(rho E - |m|^2 / (2 rho)).
* F^c_d = (m_d, m_d u + p e_d, u_d (rho E + p)).
* tau = mu (grad u + grad u^T - 2/3 div u I), constant mu (Stokes' hypothesis).
* heat flux q = -(mu gamma / ((gamma-1) Pr)) grad(p/rho)  (R cancels).
* F^v_d = (0, tau_{.d}, tau_{.d} . u - q_d).
* Lifted variables are the primitives W = (rho, u, v, w, p) ("one gradient per
  direction per primitive variable", Sec. 5.4); grad(p/rho) =
  (grad p - (p/rho) grad rho)/rho.
* Roe: Roe-averaged 5-wave flux, no entropy fix; optional Harten-type smoothing
  |lam| -> (lam^2 + delta^2)/(2 delta) for |lam| < delta, delta = 0.1 c_roe
  (makes the discrete operator C^1 for finite-difference checks of the adjoint).
* HLLC (Toro): S_L = min(u_nL - c_L, u_roe - c_roe), S_R = max(u_nR + c_R,
  u_roe + c_roe), contact speed from the jump conditions, 4-branch star flux.
* Rusanov (local Lax-Friedrichs): (F_L + F_R).n / 2 - lambda_max (U_R - U_L) / 2,
  lambda_max = max(|u_nL| + c_L, |u_nR| + c_R).

Variables are in the LAST tensor dimension (length 5); gradients are
``[..., 3 (x_d), 5 (var)]``; normals ``[..., 3]``.
"""
from __future__ import annotations

import math

import torch


class Gas:
    def __init__(self, gamma=1.4, Pr=0.72, mu=1.0 / 1600.0):
        self.gamma, self.Pr, self.mu = gamma, Pr, mu


def prim(U, gas):
    rho = U[..., 0]
    u, v, w = U[..., 1] / rho, U[..., 2] / rho, U[..., 3] / rho
    p = (gas.gamma - 1.0) * (U[..., 4] - 0.5 * rho * (u * u + v * v + w * w))
    return torch.stack([rho, u, v, w, p], dim=-1)


def cons(W, gas):
    rho, u, v, w, p = W.unbind(-1)
    E = p / (gas.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return torch.stack([rho, rho * u, rho * v, rho * w, E], dim=-1)


def flux_conv(U, W):
    """F^c as [..., 3 (d), 5]."""
    rho, u, v, w, p = W.unbind(-1)
    E = U[..., 4]
    vel = (u, v, w)
    rows = []
    for d in range(3):
        ud = vel[d]
        mom = [U[..., 1 + c] * ud + (p if c == d else 0.0) for c in range(3)]
        rows.append(torch.stack([U[..., 1 + d], mom[0], mom[1], mom[2], ud * (E + p)], dim=-1))
    return torch.stack(rows, dim=-2)


def flux_visc(W, G, gas):
    """F^v as [..., 3 (d), 5] from primitives W and their gradients G [...,3,5]."""
    rho, u, v, w, p = W.unbind(-1)
    vel = (u, v, w)
    # grad u_c along x_d: G[..., d, 1 + c]
    gu = [[G[..., d, 1 + c] for d in range(3)] for c in range(3)]  # gu[c][d] = d u_c / d x_d
    div = gu[0][0] + gu[1][1] + gu[2][2]
    lam_th = gas.mu * gas.gamma / ((gas.gamma - 1.0) * gas.Pr)
    rows = []
    for d in range(3):
        tau = [gas.mu * (gu[c][d] + gu[d][c] - (2.0 / 3.0 * div if c == d else 0.0)) for c in range(3)]
        dT = (G[..., d, 4] - (p / rho) * G[..., d, 0]) / rho  # d(p/rho)/dx_d
        energy = tau[0] * vel[0] + tau[1] * vel[1] + tau[2] * vel[2] + lam_th * dT
        rows.append(torch.stack([torch.zeros_like(rho), tau[0], tau[1], tau[2], energy], dim=-1))
    return torch.stack(rows, dim=-2)


def normal_flux(F, n):
    """sum_d F[..., d, :] n_d."""
    return (F * n.unsqueeze(-1)).sum(dim=-2)


def _euler_normal_flux(U, W, n):
    rho, u, v, w, p = W.unbind(-1)
    un = u * n[..., 0] + v * n[..., 1] + w * n[..., 2]
    return torch.stack([rho * un, U[..., 1] * un + p * n[..., 0], U[..., 2] * un + p * n[..., 1],
                        U[..., 3] * un + p * n[..., 2], (U[..., 4] + p) * un], dim=-1)


def riemann_roe(UL, UR, n, gas, smooth: bool = False):
    """Roe flux f*(U_L, U_R, n) (per unit area), frame-free form."""
    g = gas.gamma
    WL, WR = prim(UL, gas), prim(UR, gas)
    FL, FR = _euler_normal_flux(UL, WL, n), _euler_normal_flux(UR, WR, n)
    rL, rR = WL[..., 0], WR[..., 0]
    sL, sR = torch.sqrt(rL), torch.sqrt(rR)
    HL = (UL[..., 4] + WL[..., 4]) / rL
    HR = (UR[..., 4] + WR[..., 4]) / rR
    wsum = sL + sR
    vel = (sL.unsqueeze(-1) * WL[..., 1:4] + sR.unsqueeze(-1) * WR[..., 1:4]) / wsum.unsqueeze(-1)
    H = (sL * HL + sR * HR) / wsum
    q2 = (vel * vel).sum(-1)
    c = torch.sqrt((g - 1.0) * (H - 0.5 * q2))
    rho = sL * sR
    un = (vel * n).sum(-1)
    dW = WR - WL
    dp = dW[..., 4]
    dun = (dW[..., 1:4] * n).sum(-1)
    dvel = dW[..., 1:4]
    a1 = (dp - rho * c * dun) / (2 * c * c)
    a5 = (dp + rho * c * dun) / (2 * c * c)
    a2 = dW[..., 0] - dp / (c * c)
    lam1, lam2, lam5 = un - c, un, un + c

    def absf(lam):
        if not smooth:
            return torch.abs(lam)
        delta = 0.1 * c
        return torch.where(torch.abs(lam) < delta, (lam * lam + delta * delta) / (2 * delta), torch.abs(lam))

    l1, l2, l5 = absf(lam1), absf(lam2), absf(lam5)
    # eigenvectors
    one = torch.ones_like(un)
    zero = torch.zeros_like(un)
    r1 = torch.cat([one.unsqueeze(-1), vel - c.unsqueeze(-1) * n, (H - un * c).unsqueeze(-1)], dim=-1)
    r5 = torch.cat([one.unsqueeze(-1), vel + c.unsqueeze(-1) * n, (H + un * c).unsqueeze(-1)], dim=-1)
    r2 = torch.cat([one.unsqueeze(-1), vel, (0.5 * q2).unsqueeze(-1)], dim=-1)
    dvt = dvel - dun.unsqueeze(-1) * n  # tangential velocity jump
    rt = torch.cat([zero.unsqueeze(-1), dvt, (vel * dvt).sum(-1).unsqueeze(-1)], dim=-1)  # shear waves * jump
    diss = (l1 * a1).unsqueeze(-1) * r1 + (l5 * a5).unsqueeze(-1) * r5 + (l2 * a2).unsqueeze(-1) * r2 \
        + (l2 * rho).unsqueeze(-1) * rt
    return 0.5 * (FL + FR) - 0.5 * diss


def riemann_rusanov(UL, UR, n, gas):
    """Rusanov / local Lax-Friedrichs flux."""
    WL, WR = prim(UL, gas), prim(UR, gas)
    FL, FR = _euler_normal_flux(UL, WL, n), _euler_normal_flux(UR, WR, n)
    cL = torch.sqrt(gas.gamma * WL[..., 4] / WL[..., 0])
    cR = torch.sqrt(gas.gamma * WR[..., 4] / WR[..., 0])
    uL = (WL[..., 1:4] * n).sum(-1)
    uR = (WR[..., 1:4] * n).sum(-1)
    lam = torch.maximum(torch.abs(uL) + cL, torch.abs(uR) + cR)
    return 0.5 * (FL + FR) - 0.5 * lam.unsqueeze(-1) * (UR - UL)


def riemann_hllc(UL, UR, n, gas):
    """HLLC flux (Toro) with Einfeldt/Davis wave-speed estimates."""
    g = gas.gamma
    WL, WR = prim(UL, gas), prim(UR, gas)
    FL, FR = _euler_normal_flux(UL, WL, n), _euler_normal_flux(UR, WR, n)
    rL, rR = WL[..., 0], WR[..., 0]
    pL, pR = WL[..., 4], WR[..., 4]
    uL = (WL[..., 1:4] * n).sum(-1)
    uR = (WR[..., 1:4] * n).sum(-1)
    cL = torch.sqrt(g * pL / rL)
    cR = torch.sqrt(g * pR / rR)
    sL, sR = torch.sqrt(rL), torch.sqrt(rR)
    HL = (UL[..., 4] + pL) / rL
    HR = (UR[..., 4] + pR) / rR
    vel = (sL.unsqueeze(-1) * WL[..., 1:4] + sR.unsqueeze(-1) * WR[..., 1:4]) / (sL + sR).unsqueeze(-1)
    H = (sL * HL + sR * HR) / (sL + sR)
    c = torch.sqrt((g - 1.0) * (H - 0.5 * (vel * vel).sum(-1)))
    un = (vel * n).sum(-1)
    SL = torch.minimum(uL - cL, un - c)
    SR = torch.maximum(uR + cR, un + c)
    Sstar = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))

    def star(U, W, S, uN):
        rho = W[..., 0]
        fac = rho * (S - uN) / (S - Sstar)
        vt = W[..., 1:4] - uN.unsqueeze(-1) * n
        mom = fac.unsqueeze(-1) * (vt + Sstar.unsqueeze(-1) * n)
        E = fac * (U[..., 4] / rho + (Sstar - uN) * (Sstar + W[..., 4] / (rho * (S - uN))))
        return torch.cat([fac.unsqueeze(-1), mom, E.unsqueeze(-1)], dim=-1)

    FsL = FL + SL.unsqueeze(-1) * (star(UL, WL, SL, uL) - UL)
    FsR = FR + SR.unsqueeze(-1) * (star(UR, WR, SR, uR) - UR)
    e = lambda m: m.unsqueeze(-1)
    return torch.where(e(SL >= 0), FL, torch.where(e(Sstar >= 0), FsL, torch.where(e(SR >= 0), FsR, FR)))


# ---------------------------------------------------------------------------
# two-point volume fluxes of the split form (Sec. 3.3, Eq. semiDiscreteSplit)
# ---------------------------------------------------------------------------


def log_mean(a, b):
    """Logarithmic mean (a - b) / (ln a - ln b) of positive a, b in the form of
    Ismail & Roe (2009): with zeta = a/b, f = (zeta - 1)/(zeta + 1) and u = f^2,
    ln(zeta) = 2 atanh(f), so the mean is (a + b) / (2 F) with F = atanh(f)/f =
    ln(zeta)/(2 f).  For u < 1e-2 (where the quotient loses digits) F is the series
    sum_k u^k / (2k + 1), kept to u^7 (the next term is below 1e-17)."""
    zeta = a / b
    f = (zeta - 1.0) / (zeta + 1.0)
    u = f * f
    series = torch.zeros_like(u)
    for k in range(7, -1, -1):
        series = series * u + 1.0 / (2 * k + 1)
    safe_f = torch.where(u < 1e-2, torch.ones_like(f), f)
    F = torch.where(u < 1e-2, series, torch.log(zeta) / (2.0 * safe_f))
    return (a + b) / (2.0 * F)


def two_point_contravariant(Ua, Wa, Ub, Wb, Ja_a, Ja_b, kind: str, gamma: float = 1.4):
    """Contravariant two-point flux sum_d F#_d(U_a, U_b) * (Ja_d(a) + Ja_d(b)) / 2.

    kind "pirozzoli": kinetic-energy-preserving flux of Pirozzoli (2011), the one
    of the paper's NACA 64418 computation (Sec. 7.1): with arithmetic means {.},
    F#_rho = {rho}{u_d}, F#_m = {rho}{u_d}{u} + {p} e_d, F#_E = {rho}{u_d}{H},
    H = (rho E + p) / rho.  kind "chandrashekar": the entropy-conservative flux of
    Chandrashekar (2013) with beta = rho / (2 p), logarithmic means rho_ln, beta_ln:
    F#_rho = rho_ln {u_d}, F#_m = F#_rho {u} + ({rho} / (2 {beta})) e_d,
    F#_E = F#_rho (1 / (2 (gamma - 1) beta_ln) - {|u|^2} / 2) + {u} . F#_m.
    kind "central": (F(U_a) + F(U_b)) / 2 (standard DG).
    Variables last; Ja_* are [..., 3] (the row Ja^l_. of the sweep direction l).
    """
    Jm = 0.5 * (Ja_a + Ja_b)
    if kind == "central":
        Fa = flux_conv(Ua, Wa)  # [..., 3, 5]
        Fb = flux_conv(Ub, Wb)
        return 0.5 * ((Fa + Fb) * Jm.unsqueeze(-1)).sum(-2)
    if kind == "chandrashekar":
        ra, rb = Wa[..., 0], Wb[..., 0]
        ba, bb = ra / (2.0 * Wa[..., 4]), rb / (2.0 * Wb[..., 4])
        vel = 0.5 * (Wa[..., 1:4] + Wb[..., 1:4])
        q2 = 0.5 * ((Wa[..., 1:4] ** 2).sum(-1) + (Wb[..., 1:4] ** 2).sum(-1))
        ptil = 0.5 * (ra + rb) / (ba + bb)
        frho = log_mean(ra, rb) * (vel * Jm).sum(-1)
        fm = frho.unsqueeze(-1) * vel + ptil.unsqueeze(-1) * Jm
        fE = frho * (1.0 / (2.0 * (gamma - 1.0) * log_mean(ba, bb)) - 0.5 * q2) + (vel * fm).sum(-1)
        return torch.cat([frho.unsqueeze(-1), fm, fE.unsqueeze(-1)], dim=-1)
    rho = 0.5 * (Wa[..., 0] + Wb[..., 0])
    vel = 0.5 * (Wa[..., 1:4] + Wb[..., 1:4])
    p = 0.5 * (Wa[..., 4] + Wb[..., 4])
    Ha = (Ua[..., 4] + Wa[..., 4]) / Wa[..., 0]
    Hb = (Ub[..., 4] + Wb[..., 4]) / Wb[..., 0]
    H = 0.5 * (Ha + Hb)
    uc = (vel * Jm).sum(-1)  # contravariant mean velocity
    m = rho * uc
    return torch.cat([m.unsqueeze(-1), m.unsqueeze(-1) * vel + p.unsqueeze(-1) * Jm, (m * H).unsqueeze(-1)], dim=-1)


# ---------------------------------------------------------------------------
# exact solutions used as Dirichlet data and source terms (Sec. 2.2 names
# Dirichlet boundaries; the fields themselves are the test cases' definitions)
# ---------------------------------------------------------------------------

EXACT_TGV, EXACT_FREESTREAM, EXACT_MANUFACTURED = 0, 1, 2


def exact_state(kind: int, x, t: float, gas, Ma: float = 0.1):
    """Conservative state [..., 5] at points x [..., 3] and time t."""
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    if kind == EXACT_TGV:
        u = torch.sin(X) * torch.cos(Y) * torch.cos(Z)
        v = -torch.cos(X) * torch.sin(Y) * torch.cos(Z)
        w = torch.zeros_like(u)
        p = 1.0 / (gas.gamma * Ma * Ma) + (torch.cos(2 * X) + torch.cos(2 * Y)) * (torch.cos(2 * Z) + 2.0) / 16.0
        return cons(torch.stack([torch.ones_like(u), u, v, w, p], -1), gas)
    if kind == EXACT_FREESTREAM:
        one = torch.ones_like(X)
        return cons(torch.stack([one, 0.3 * one, 0.2 * one, 0.1 * one, one / gas.gamma], -1), gas)
    if kind == EXACT_MANUFACTURED:
        rho = 2.0 + 0.1 * torch.sin(math.pi * (X + Y + Z - 2.0 * t))
        return torch.stack([rho, rho, rho, rho, rho * rho], -1)
    raise ValueError(kind)


def manufactured_source(x, t: float, gas):
    """S = U_t + div(F^c(U) - F^v(U, grad U)) for the manufactured field.

    Obtained by exact forward-mode automatic differentiation (torch.func) of
    the closed form, point by point; no hand derivation is involved.
    """
    from torch.func import jacfwd, vmap

    shape = x.shape[:-1]
    pts = x.detach().reshape(-1, 3)

    def U_of(xt):  # xt: [4] = (x, y, z, t)
        return exact_state(EXACT_MANUFACTURED, xt[:3], xt[3], gas)

    def W_of(xt):
        return prim(U_of(xt), gas)

    def flux_total(xt):
        U = U_of(xt)
        W = prim(U, gas)
        G = jacfwd(W_of)(xt)[:, :3].T  # [3 (d), 5]
        return flux_conv(U, W) - flux_visc(W, G, gas)  # [3, 5]

    def S_of(xt):
        dUdt = jacfwd(U_of)(xt)[:, 3]
        dF = jacfwd(flux_total)(xt)  # [3 (d), 5, 4]
        return dUdt + dF[0, :, 0] + dF[1, :, 1] + dF[2, :, 2]

    tt = torch.full((pts.shape[0], 1), float(t), dtype=pts.dtype)
    S = vmap(S_of)(torch.cat([pts, tt], dim=1))
    return S.reshape(*shape, 5)
