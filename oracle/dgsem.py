"""DGSEM semi-discrete operator, LSERK4(5) and the discrete adjoint (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The right-hand side follows, step by step:

  a1  prolongation of U to the faces: U^{+xi1}_{mn} = sum_o U_{mno} l_o(1)
      (Sec. 3.1, "Surface integral"); the face primitives are W(U_face);
  a2  BR1 surface value U* = (U_L + U_R)/2 in the lifted (primitive) variables
      (Sec. 3.1, "Approximation for second order equations");
  a3  lifting, Eq. discreteGradient:
      g^d_ijk = (1/J_ijk)[ sum_a Dhat_ia Ucal^{1,d}_ajk + (l_hat(+-1) U* n_d s)
                 + ... (3 directions) ],  Ucal^{l,d} = Ja^l_d W;
  a4  prolongation of g to the faces (same operator as a1);
  a5  numerical flux on every side, computed once in the master's normal:
      f* s = [f*_Riemann(U_L, U_R, n) - (F^v(W_L,g_L) + F^v(W_R,g_R)).n / 2] s,
      the slave uses -f* s (Sec. 5.1, 5.5);
  a6  volume fluxes F = F^c - F^v and contravariant fluxes Fcal^l = sum_d Ja^l_d F^d;
  a7  volume integral sum_a Fcal^1_ajk Dhat_ia + (directions 2, 3);
  a8  surface integral [f* s] l_hat(+-1) on the six faces;
  a9  U_t = -(a7 + a8) / J  (Eq. semiDiscrete).

Boundary sides (Dirichlet, Sec. 2.2): U_R = exact state at the face nodes, used
in both the Riemann flux and the BR1 mean; g_R = g_L.

Time integration (Sec. 3.4): Williamson two-register low-storage RK, with the
five-stage fourth-order coefficients of Carpenter & Kennedy (1994).  The paper
prints no coefficients; the published ones are used and pinned by the order
conditions in the tests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import equations as eq
from .basis import DT, Basis
from .mesh import MeshGeometry, apply_dir, prolong, spread

# Carpenter & Kennedy (1994), 4th order, 5 stages, 2N storage
RK_A = [0.0,
        -567301805773.0 / 1357537059087.0,
        -2404267990393.0 / 2016746695238.0,
        -3550918686646.0 / 2091501179385.0,
        -1275806237668.0 / 842570457699.0]
RK_B = [1432997174477.0 / 9575080441755.0,
        5161836677717.0 / 13612068292357.0,
        1720146321549.0 / 2090206949498.0,
        3134564353537.0 / 4481467310338.0,
        2277821191437.0 / 14882151754819.0]
RK_C = [0.0,
        1432997174477.0 / 9575080441755.0,
        2526269341429.0 / 6820363962896.0,
        2006345519317.0 / 3224310063776.0,
        2802321613138.0 / 2924317926251.0]

ROE, HLLC, RUSANOV = 0, 1, 3
EC = 4  # entropy-conservative surface flux: Chandrashekar's two-point flux in the face normal
# boundary conditions (Sec. 2.2 names Dirichlet, inflow/outflow and wall conditions, imposed
# weakly through the outer state of the numerical flux): the outer state U_R is the exact
# solution, the inner state (outflow: extrapolation), or the inner state with its normal
# velocity reversed (slip wall); every kind takes the inner lifted gradients, g_R = g_L
BC_EXACT, BC_OUTFLOW, BC_SLIP_WALL = 0, 1, 2


@dataclass
class Params:
    N: int = 3
    node_type: int = 0  # 0 LG, 1 LGL
    riemann: int = ROE
    smooth_roe: bool = False
    gamma: float = 1.4
    Pr: float = 0.72
    mu: float = 1.0 / 1600.0
    Ma: float = 0.1  # for the TGV exact state used as boundary data
    bc_exact: object = eq.EXACT_TGV  # exact function id (or callable (x, t) -> U) on Dirichlet sides
    source: bool = False  # manufactured-solution source term
    split: str = ""  # "" standard weak form; "pirozzoli" / "chandrashekar" / "central": split form (LGL only)
    bc_kinds: dict = None  # boundary id -> BC_EXACT (default), BC_OUTFLOW, BC_SLIP_WALL
    lifting: str = "br1"  # "br1" (Eq. discreteGradient) or "br2" (face gradients of Bassi & Rebay 1997)
    eta_br2: float = 2.0  # BR2 penalty factor on a face's own lifting


class DGSEM:
    def __init__(self, params: Params, coords: np.ndarray, conn: np.ndarray, mortars=None):
        self.p = params
        self.b = Basis(params.N, params.node_type)
        self.geo = MeshGeometry(self.b, coords, conn, mortars)
        self.gas = eq.Gas(params.gamma, params.Pr, params.mu)
        self.K, self.n = self.geo.K, self.b.n

    # ------------------------------------------------------------------
    def _riemann(self, UL, UR, nv):
        if self.p.riemann == ROE:
            return eq.riemann_roe(UL, UR, nv, self.gas, smooth=self.p.smooth_roe)
        if self.p.riemann == RUSANOV:
            return eq.riemann_rusanov(UL, UR, nv, self.gas)
        if self.p.riemann == EC:
            return eq.two_point_contravariant(UL, eq.prim(UL, self.gas), UR, eq.prim(UR, self.gas), nv, nv,
                                              "chandrashekar", self.gas.gamma)
        return eq.riemann_hllc(UL, UR, nv, self.gas)

    def rhs(self, U: torch.Tensor, t: float = 0.0, parts: bool = False):
        """U: [K, 5, n, n, n] float64 -> U_t of the same shape."""
        geo, b, gas = self.geo, self.b, self.gas
        K, n = self.K, self.n
        J = geo.J.unsqueeze(1)  # [K,1,n,n,n]
        Ja = geo.Ja
        W = eq.prim(U.movedim(1, -1), gas).movedim(-1, 1)  # [K,5,n,n,n]

        # a1: face states
        Uf = geo.face_values(U, b.l_side)  # [K,6,5,q,p]
        Wf = eq.prim(Uf.movedim(2, -1), gas).movedim(-1, 2)
        UL, UR = geo.master_slave(Uf)
        WL, WR = geo.master_slave(Wf)
        if len(geo.virt) > 0:  # mortar sides interpolate the solution U; W follows from it
            WR = WR.clone()
            WR[geo.virt] = eq.prim(UR[geo.virt].movedim(1, -1), gas).movedim(-1, 1)
        bnd = geo.bnd
        if len(bnd) > 0:
            xb = geo.xface[bnd].movedim(1, -1)
            if callable(self.p.bc_exact):
                Ub = self.p.bc_exact(xb, t)
            else:
                Ub = eq.exact_state(self.p.bc_exact, xb, t, gas, self.p.Ma)
            kinds = self.p.bc_kinds or {}
            kind = torch.tensor([kinds.get(int(geo.bc[sd]), BC_EXACT) for sd in bnd.tolist()])
            Ui = UL[bnd].movedim(1, -1)  # [B,q,p,5] inner state
            nb = geo.nvec[bnd].movedim(1, -1)  # [B,q,p,3] outward normal of the element
            mn = (Ui[..., 1:4] * nb).sum(-1, keepdim=True)
            Umirror = torch.cat([Ui[..., :1], Ui[..., 1:4] - 2.0 * mn * nb, Ui[..., 4:]], dim=-1)
            k = kind.view(-1, 1, 1, 1)
            Ub = torch.where(k == BC_OUTFLOW, Ui, torch.where(k == BC_SLIP_WALL, Umirror, Ub))
            UR = UR.clone(); WR = WR.clone()
            UR[bnd] = Ub.movedim(-1, 1)
            WR[bnd] = eq.prim(Ub, gas).movedim(-1, 1)

        # a2, a3: BR1 lifting
        Wstar = 0.5 * (WL + WR)  # [S,5,q,p]
        nS = geo.nvec * geo.sarea.unsqueeze(1)  # [S,3,q,p], master outward n s
        Qm = (Wstar.unsqueeze(2) * nS.unsqueeze(1)).flatten(1, 2)  # [S,15,q,p] (var, d)
        Qf = geo.to_elements(Qm, -Qm).view(K, 6, 5, 3, n, n)  # slave: outward normal is -n
        grads = []
        for d in range(3):
            acc = torch.zeros_like(W)
            for l in range(3):
                acc = acc + apply_dir(b.Dhat, Ja[:, l, d].unsqueeze(1) * W, l)
            for s in range(6):
                l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
                acc = acc + spread(Qf[:, s, :, d], b.lhat_side(sgn), l)
            grads.append(acc / J)
        G = torch.stack(grads, dim=1)  # [K, 3 (d), 5, n,n,n]

        # a4: gradients on the faces
        if self.p.lifting == "br2":
            Gf = self._br2_face_gradients(G, Wf, Qf)
        else:
            Gf = geo.face_values(G.flatten(1, 2), b.l_side)  # [K,6,15,q,p]
        GL, GR = geo.master_slave(Gf)
        if len(bnd) > 0:
            GR = GR.clone()
            GR[bnd] = GL[bnd]

        # a5: numerical flux on the sides (master normal), times s
        nv = geo.nvec.movedim(1, -1)  # [S,q,p,3]
        mv = lambda A: A.movedim(1, -1)
        gv = lambda A: A.view(A.shape[0], 3, 5, n, n).permute(0, 3, 4, 1, 2)  # [S,q,p,3,5]
        fc = self._riemann(mv(UL), mv(UR), nv)
        fv = 0.5 * (eq.normal_flux(eq.flux_visc(mv(WL), gv(GL), gas), nv)
                    + eq.normal_flux(eq.flux_visc(mv(WR), gv(GR), gas), nv))
        fstar = ((fc - fv) * geo.sarea.unsqueeze(-1)).movedim(-1, 1)  # [S,5,q,p]

        # a6, a7: volume integral
        Uv, Wv = U.movedim(1, -1), W.movedim(1, -1)
        Gv = G.permute(0, 3, 4, 5, 1, 2)  # [K,n,n,n,3,5]
        Ff = geo.to_elements(fstar, -fstar)  # [K,6,5,q,p] outward f* s of every element face
        if self.p.split:
            vol, surf = self._split_form(U, Uv, Wv, Gv, Ff)
        else:
            F = eq.flux_conv(Uv, Wv) - eq.flux_visc(Wv, Gv, gas)  # [K,n,n,n,3,5]
            vol = torch.zeros_like(U)
            for l in range(3):
                Fl = sum(Ja[:, l, d].unsqueeze(-1) * F[..., d, :] for d in range(3))  # [K,n,n,n,5]
                vol = vol + apply_dir(b.Dhat, Fl.movedim(-1, 1), l)

            # a8: surface integral
            surf = torch.zeros_like(U)
            for s in range(6):
                l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
                surf = surf + spread(Ff[:, s], b.lhat_side(sgn), l)

        # a9
        Ut = -(vol + surf) / J
        if self.p.source:
            Ut = Ut + self.source(t)
        if parts:
            return Ut, dict(W=W, G=G, fstar=fstar, vol=vol, surf=surf, Wstar=Wstar, UL=UL, UR=UR, GL=GL, GR=GR)
        return Ut

    def _br2_face_gradients(self, G, Wf, Qf):
        """BR2 face gradients (Bassi & Rebay 1997; the paper names BR2 without formulas).
        Reading: the BR1 gradient G of Eq. discreteGradient is the broken gradient plus the
        lifting r_f of every face, r_f = (1/J) l_hat(+-1) (U* - U_e) n s_hat spread along the
        face's direction, with U_e the element's own face state and n s_hat its own outward
        metric (Ja^l . N).  On each side of a face the viscous flux takes
        (G - sum_f' r_f') + eta r_f, traced to the face; the volume integral keeps G."""
        geo, b = self.geo, self.b
        K, n = self.K, self.n
        J = geo.J.unsqueeze(1).unsqueeze(1)  # [K,1,1,n,n,n]
        r = []
        for s in range(6):
            l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
            n_own = sgn * prolong(geo.Ja[:, l], b.l_side(sgn), l)  # [K,3 (d),q,p]
            jump = Qf[:, s] - Wf[:, s].unsqueeze(2) * n_own.unsqueeze(1)  # [K,5,3,q,p]
            rs = torch.stack([spread(jump[:, :, d], b.lhat_side(sgn), l) for d in range(3)], dim=1)  # [K,3,5,...]
            r.append(rs / J)
        broken = G - sum(r)
        out = []
        for s in range(6):
            l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
            face = prolong((broken + self.p.eta_br2 * r[s]).flatten(1, 2), b.l_side(sgn), l)
            out.append(face)
        return torch.stack(out, dim=1)  # [K,6,15,q,p]

    def _split_form(self, U, Uv, Wv, Gv, Ff):
        """Split-form volume and surface terms (Sec. 3.3, Eq. semiDiscreteSplit) on
        Gauss-Lobatto nodes: advective volume term 2 sum_a D_ia Fcal#^l(U_i, U_a)
        with metric-averaged two-point fluxes, viscous volume term in strong form
        -sum_l D^(l) Fcal^{v,l}, and the strong-form surface penalty
        l_hat(+-1) [f* s - Fcal.N] with the outward reference normal N = +-1 and
        Fcal the element's own total contravariant flux on the face."""
        if self.p.node_type != 1:
            raise ValueError("the split form needs Gauss-Lobatto nodes (summation by parts)")
        geo, b, gas = self.geo, self.b, self.gas
        Ja = geo.Ja
        Fc = eq.flux_conv(Uv, Wv)
        Fv = eq.flux_visc(Wv, Gv, gas)
        vol = torch.zeros_like(U)
        surf = torch.zeros_like(U)
        for l in range(3):
            Jl = Ja[:, l].movedim(1, -1)  # [K,n,n,n,3] row Ja^l_.
            # two-point fluxes along lines of direction l: axis 3 - l of [K,k,j,i]
            ax = 3 - l
            ul, wl, jl = Uv.movedim(ax, -2), Wv.movedim(ax, -2), Jl.movedim(ax, -2)  # [..., n(line), 5]
            Fs = eq.two_point_contravariant(ul.unsqueeze(-2), wl.unsqueeze(-2), ul.unsqueeze(-3), wl.unsqueeze(-3),
                                            jl.unsqueeze(-2), jl.unsqueeze(-3), self.p.split,
                                            gas.gamma)  # [..., i, a, 5]
            adv = 2.0 * torch.einsum("ia,...iav->...iv", b.D, Fs)
            vol = vol + adv.movedim(-2, ax).movedim(-1, 1)
            Fvl = sum(Ja[:, l, d].unsqueeze(-1) * Fv[..., d, :] for d in range(3)).movedim(-1, 1)
            Fcl = sum(Ja[:, l, d].unsqueeze(-1) * Fc[..., d, :] for d in range(3)).movedim(-1, 1)
            vol = vol - apply_dir(b.D, Fvl, l)
            for sgn in (-1, 1):
                s = 2 * l + (0 if sgn < 0 else 1)
                interior = prolong(Fcl - Fvl, b.l_side(sgn), l)  # [K,5,q,p]
                surf = surf + spread(Ff[:, s] - sgn * interior, b.lhat_side(sgn), l)
        return vol, surf

    def source(self, t: float) -> torch.Tensor:
        x = self.geo.x.movedim(1, -1)  # [K,n,n,n,3]
        S = eq.manufactured_source(x, t, self.gas)
        return S.view(self.K, self.n, self.n, self.n, 5).movedim(-1, 1)

    # ------------------------------------------------------------------
    def rk_step(self, U, dU, t, dt, stages_out=None):
        """One LSERK4(5) step (Williamson 2N form): dU = A_k dU + dt L(U, t + c_k dt);
        U = U + B_k dU."""
        for k in range(5):
            if stages_out is not None:
                stages_out.append(U.clone())
            Ut = self.rhs(U, t + RK_C[k] * dt)
            dU = RK_A[k] * dU + dt * Ut
            U = U + RK_B[k] * dU
        return U, dU

    def run(self, U, nsteps, dt, t0=0.0):
        dU = torch.zeros_like(U)
        t = t0
        for _ in range(nsteps):
            U, dU = self.rk_step(U, dU, t, dt)
            t += dt
        return U

    # ------------------------------------------------------------------
    def quad_weights(self) -> torch.Tensor:
        """omega_i omega_j omega_k J at every node, [K, n, n, n]."""
        w = self.b.w
        w3 = w.view(-1, 1, 1) * w.view(1, -1, 1) * w.view(1, 1, -1)
        return self.geo.J * w3

    def integrals(self, U) -> torch.Tensor:
        """Conserved totals (5) and kinetic energy, by the collocated quadrature."""
        wJ = self.quad_weights().unsqueeze(1)
        tot = (wJ * U).sum(dim=(0, 2, 3, 4))
        ke = (self.quad_weights() * 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2) / U[:, 0]).sum()
        return torch.cat([tot, ke.view(1)])

    def kinetic_energy(self, U) -> torch.Tensor:
        return (self.quad_weights() * 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2) / U[:, 0]).sum()

    def dt_max(self, U, cfl: float = 0.9, dfl: float = 0.9) -> float:
        """Time step from Eqs. CFLCondition and DFLCondition, evaluated per
        reference direction through the metrics (reading: gamma_RK = 1,
        reference element length 2, directional rates summed)."""
        gas, N = self.gas, self.p.N
        W = eq.prim(U.movedim(1, -1), gas)
        rho, vel, p = W[..., 0], W[..., 1:4], W[..., 4]
        c = torch.sqrt(gas.gamma * p / rho)
        J = self.geo.J
        lam_c = torch.zeros_like(rho)
        lam_v = torch.zeros_like(rho)
        kv = max(4.0 / 3.0, gas.gamma / gas.Pr) * gas.mu / rho
        for l in range(3):
            Ja = self.geo.Ja[:, l].movedim(1, -1)  # [K,n,n,n,3]
            nrm = torch.sqrt((Ja * Ja).sum(-1))
            lam_c = lam_c + (torch.abs((Ja * vel).sum(-1)) + c * nrm) / J
            lam_v = lam_v + kv * (nrm / J) ** 2
        dtc = cfl * 2.0 / ((2 * N + 1) * lam_c.max())
        dtv = dfl * 4.0 / ((2 * N + 1) * lam_v.max()) if gas.mu > 0 else torch.tensor(float("inf"))
        return float(torch.minimum(dtc, dtv))

    # ------------------------------------------------------------------
    # discrete adjoint
    def rhs_vjp(self, U, t, lam):
        """(d RHS / d U)^T lam by reverse-mode differentiation of this oracle."""
        with torch.enable_grad():
            Ux = U.detach().clone().requires_grad_(True)
            Ut = self.rhs(Ux, t)
            (g,) = torch.autograd.grad(Ut, Ux, lam)
        return g

    def adjoint_step(self, stages, lamU, lam_dU, t, dt):
        """Reverse of one rk_step, given its five stage inputs."""
        for k in reversed(range(5)):
            lam_dU = lam_dU + RK_B[k] * lamU
            lamU = lamU + dt * self.rhs_vjp(stages[k], t + RK_C[k] * dt, lam_dU)
            lam_dU = RK_A[k] * lam_dU
        return lamU, lam_dU

    def gradient_ke(self, U0, nsteps, dt, t0=0.0):
        """dJ/dU0 for J = kinetic energy at the final time (sweeps forward, storing
        all stage inputs, then runs the adjoint steps backwards)."""
        U, dU = U0.clone(), torch.zeros_like(U0)
        history = []
        t = t0
        for _ in range(nsteps):
            st = []
            U, dU = self.rk_step(U, dU, t, dt, stages_out=st)
            history.append((st, t))
            t += dt
        with torch.enable_grad():
            Ux = U.detach().clone().requires_grad_(True)
            Jv = self.kinetic_energy(Ux)
            (lamU,) = torch.autograd.grad(Jv, Ux)
        lam_dU = torch.zeros_like(lamU)
        for st, ts in reversed(history):
            lamU, lam_dU = self.adjoint_step(st, lamU, lam_dU, ts, dt)
        return float(Jv.detach()), lamU
