"""Mesh geometry and connectivity for the oracle (test infrastructure only).

* Mapping of each element from the reference cube (Sec. 3.1): the node
  coordinates given at (Ngeo+1)^3 Gauss-Lobatto points are interpolated to the
  solution nodes (Lagrange interpolation, exact for Ngeo <= N).
* Jacobian J = det(grad_xi x) (Sec. 3.1).
* Metric terms in curl form, Eq. contravariantBasisVectorsCurl:
  Ja^i_n = -xhat_i . curl_xi(x_l grad_xi x_m), (n, m, l) cyclic.  Reading: the
  product x_l grad_xi x_m is collocated on the degree-N Gauss-Lobatto points and
  differentiated there with their D matrix; the resulting degree-N polynomial
  is interpolated to the solution nodes.  This keeps the discrete metric
  identities exact and makes the face metrics of the two elements sharing a
  side agree, which free-stream preservation (Sec. 3.1) needs on LG nodes.
* Face normal and surface element (Sec. 3.1, "Surface integral"):
  ntilde_d = sum_i Ja^i_d Nref^i, s_hat = |ntilde|, n_hat = ntilde / s_hat,
  with Ja taken as the interpolation of the master element's volume metrics to
  the face.
* Sides, master/slave and flip (Sec. 5.1): a side is stored once, in the
  side-local frame of its master element; the slave's face data are mapped
  with the orientation code given in the connectivity.
* Mortars (Sec. "Non-conforming meshes"): every small side of a non-conforming
  interface is a side of its own whose master is the small element and whose
  "slave" values are interpolated from the big element's face (I^a along each
  cut direction of the big side); values returned to the big element are the
  L2 projection (P^a) of the slave values of its small sides.  Mortar sides
  carry bc = -2.

Index conventions are those of the ``workloads`` module docstring.
"""
from __future__ import annotations

import numpy as np
import torch

from .basis import DT, Basis, diff_matrix, lagrange_matrix, lobatto_nodes


def apply_dir(M: torch.Tensor, f: torch.Tensor, l: int) -> torch.Tensor:
    """Apply the 1-D matrix M along reference direction l of f[..., k, j, i]:
    out[.., a, ..] = sum_b M[a, b] f[.., b, ..]."""
    axis = f.dim() - 1 - l
    out = torch.tensordot(f.movedim(axis, -1), M, dims=([-1], [1]))
    return out.movedim(-1, axis)


def prolong(f: torch.Tensor, lvec: torch.Tensor, l: int) -> torch.Tensor:
    """Evaluate f[..., k, j, i] on a face of direction l with weights lvec
    (the Lagrange values l_j(+-1)).  Result is [..., q, p] in side-local order."""
    axis = f.dim() - 1 - l
    return torch.tensordot(f.movedim(axis, -1), lvec, dims=([-1], [0]))


def spread(face: torch.Tensor, lvec: torch.Tensor, l: int) -> torch.Tensor:
    """Inverse layout of ``prolong``: out[..., k, j, i] = lvec[index_l] * face[..., q, p]."""
    n = lvec.shape[0]
    if l == 0:  # (q, p) = (k, j)
        return face.unsqueeze(-1) * lvec.view(1, 1, n)
    if l == 1:  # (q, p) = (k, i)
        return face.unsqueeze(-2) * lvec.view(1, n, 1)
    return face.unsqueeze(-3) * lvec.view(n, 1, 1)  # (q, p) = (j, i)


def orient_index(o: int, N: int) -> np.ndarray:
    """Flat gather index g with B.flat[q' n + p'] = A.flat[g[q' n + p']] where
    (p', q') = T_o(p, q) is the neighbour-frame position of local node (p, q)."""
    n = N + 1
    g = np.zeros(n * n, dtype=np.int64)
    for q in range(n):
        for p in range(n):
            a, b = (q, p) if o & 1 else (p, q)
            pp = N - a if o & 2 else a
            qq = N - b if o & 4 else b
            g[qq * n + pp] = q * n + p
    return g


MORTAR = -(1 << 30)  # connectivity value of a side on a mortar interface


class MeshGeometry:
    def __init__(self, basis: Basis, coords: np.ndarray, conn: np.ndarray, mortars=None):
        N, n = basis.N, basis.n
        self.basis = basis
        K = coords.shape[0]
        self.K = K
        ng = coords.shape[1]
        xgeo, _ = lobatto_nodes(ng - 1)
        X0 = torch.tensor(coords, dtype=DT).permute(0, 4, 1, 2, 3)  # [K, 3, kg, jg, ig]

        def interp(f, x_from, x_to):
            V = torch.tensor(lagrange_matrix(x_from, x_to), dtype=DT)
            for l in range(3):
                f = apply_dir(V, f, l)
            return f

        X = interp(X0, xgeo, basis.x_np)
        self.x = X  # [K, 3, n, n, n] at the solution nodes
        # The metric terms and J are invariant under a translation of the mapping
        # (grad_xi of a constant vanishes, and curl_xi(c grad_xi x_m) = 0 because the
        # tensor-product derivatives along different directions commute), so they
        # are formed from each element's coordinates relative to its first geometry
        # node: differentiating absolute coordinates that are large compared with
        # the element's width would cancel digits in every sum.
        X0r = X0 - X0[:, :, :1, :1, :1]
        D = basis.D
        # dx[e, c, l, k, j, i] = d x_c / d xi_l at the solution nodes
        Xr = interp(X0r, xgeo, basis.x_np)
        dx = torch.stack([apply_dir(D, Xr, l) for l in range(3)], dim=2)
        Jm = dx.permute(0, 3, 4, 5, 1, 2)  # [K, k, j, i, c, l]
        self.J = torch.linalg.det(Jm)
        # curl form metrics, collocated on the degree-N Lobatto points (whose
        # face nodes see only face data, so both elements of a side get the same
        # face metrics), then interpolated (exactly, degree N) to the solution nodes
        xl, _ = lobatto_nodes(N)
        Dl = torch.tensor(diff_matrix(xl), dtype=DT)
        XL = interp(X0r, xgeo, xl)
        dxl = torch.stack([apply_dir(Dl, XL, l) for l in range(3)], dim=2)
        JaL = torch.zeros(K, 3, 3, n, n, n, dtype=DT)
        for nn in range(3):
            m, ll = (nn + 1) % 3, (nn + 2) % 3
            v = [XL[:, ll] * dxl[:, m, j] for j in range(3)]  # v_j = x_l d x_m / d xi_j
            for i in range(3):
                i1, i2 = (i + 1) % 3, (i + 2) % 3
                curl_i = apply_dir(Dl, v[i2], i1) - apply_dir(Dl, v[i1], i2)
                JaL[:, i, nn] = -curl_i
        Ja = interp(JaL.flatten(1, 2), xl, basis.x_np).view(K, 3, 3, n, n, n)
        self.Ja = Ja  # [K, i(contravariant), n(physical), k, j, i]
        self._build_sides(conn, N, mortars)
        self._face_geometry()

    # ------------------------------------------------------------------
    def _build_sides(self, conn, N, mortars):
        K = self.K
        seen = {}
        m_el, m_sd, s_el, s_sd, s_or, bc = [], [], [], [], [], []
        for e in range(K):
            for s in range(6):
                nb, ns, o = (int(v) for v in conn[e, s])
                if nb == MORTAR:
                    continue
                if nb < 0:
                    m_el.append(e); m_sd.append(s); s_el.append(-1); s_sd.append(-1); s_or.append(0); bc.append(-1 - nb)
                    continue
                key = (min(e * 6 + s, nb * 6 + ns), max(e * 6 + s, nb * 6 + ns))
                if key in seen:
                    continue
                seen[key] = True
                if e * 6 + s < nb * 6 + ns:  # master = smaller (element, side) key
                    m_el.append(e); m_sd.append(s); s_el.append(nb); s_sd.append(ns)
                    s_or.append(int(conn[nb, ns, 2]))  # slave-local -> master-local
                else:
                    m_el.append(nb); m_sd.append(ns); s_el.append(e); s_sd.append(s); s_or.append(o)
                bc.append(-1)
        # mortar sides: (big element, big side, type, position a, b) per small side
        self.mortar = []
        for row in (np.zeros((0, 15), dtype=np.int64) if mortars is None else np.asarray(mortars)):
            eB, sB, typ = int(row[0]), int(row[1]), int(row[2])
            for pos in range(4):
                e2, s2, o2 = (int(v) for v in row[3 + 3 * pos:6 + 3 * pos])
                if e2 < 0:
                    continue
                a = pos % 2 if typ == 3 else (pos if typ == 1 else 0)
                b = pos // 2 if typ == 3 else (pos if typ == 2 else 0)
                self.mortar.append((len(m_el), eB, sB, typ, a, b))
                m_el.append(e2); m_sd.append(s2); s_el.append(-1); s_sd.append(-1); s_or.append(o2); bc.append(-2)
        t = lambda a: torch.tensor(a, dtype=torch.long)
        self.m_el, self.m_sd, self.s_el, self.s_sd = t(m_el), t(m_sd), t(s_el), t(s_sd)
        self.s_or = np.array(s_or)
        self.bc = t(bc)
        self.nsides = len(m_el)
        self.inner = torch.nonzero(self.bc == -1).flatten()
        self.bnd = torch.nonzero(self.bc >= 0).flatten()
        self.virt = torch.nonzero(self.bc == -2).flatten()
        n = N + 1
        # per inner side: gather index slave-local -> master frame, and its inverse
        self.to_master = torch.zeros(self.nsides, n * n, dtype=torch.long)
        self.to_slave = torch.zeros(self.nsides, n * n, dtype=torch.long)
        for sd in range(self.nsides):
            g = orient_index(int(self.s_or[sd]), N)
            self.to_master[sd] = torch.tensor(g)
            inv = np.empty_like(g)
            inv[g] = np.arange(n * n)
            self.to_slave[sd] = torch.tensor(inv)

    def _face_geometry(self):
        b = self.basis
        nvec, sarea, xf = [], [], []
        for sd in range(self.nsides):
            e, s = int(self.m_el[sd]), int(self.m_sd[sd])
            l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
            Ja_f = prolong(self.Ja[e, l], b.l_side(sgn), l)  # [3 (d), q, p]
            nt = sgn * Ja_f
            sa = torch.sqrt((nt * nt).sum(0))
            nvec.append(nt / sa)
            sarea.append(sa)
            xf.append(prolong(self.x[e], b.l_side(sgn), l))
        self.nvec = torch.stack(nvec)  # [S, 3, q, p]
        self.sarea = torch.stack(sarea)  # [S, q, p]
        self.xface = torch.stack(xf)  # [S, 3, q, p]

    # ------------------------------------------------------------------
    def face_values(self, f: torch.Tensor, lvec_of_sign) -> torch.Tensor:
        """All 6 local faces of every element: f[K, C, k, j, i] -> [K, 6, C, q, p]."""
        out = []
        for s in range(6):
            l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
            out.append(prolong(f, lvec_of_sign(sgn), l))
        return torch.stack(out, dim=1)

    def master_slave(self, faces: torch.Tensor):
        """From per-element face data [K, 6, C, q, p], return (master, slave) side
        arrays [S, C, q, p] in the master frame (slave entries of boundary sides
        are left as zeros)."""
        n = self.basis.n
        M = faces[self.m_el, self.m_sd]
        S = torch.zeros_like(M)
        inn = self.inner
        sl = faces[self.s_el[inn], self.s_sd[inn]].flatten(-2)  # [Si, C, n*n] slave-local
        idx = self.to_master[inn].unsqueeze(1).expand(-1, sl.shape[1], -1)
        S[inn] = torch.gather(sl, 2, idx).view(-1, sl.shape[1], n, n)
        b = self.basis
        for sd, eB, sB, typ, a, bq in self.mortar:
            big = faces[eB, sB]  # [C, q, p] in the big side's frame
            if typ in (1, 3):  # cut along p: interpolate along p
                big = torch.einsum("im,cqm->cqi", b.I_mortar[a], big)
            if typ in (2, 3):  # cut along q
                big = torch.einsum("jn,cnp->cjp", b.I_mortar[bq], big)
            # sub-square frame -> frame of the small side (its master)
            S[sd] = big.flatten(-2)[:, self.to_slave[sd]].view(-1, n, n)
        return M, S

    def to_elements(self, master_vals: torch.Tensor, slave_vals: torch.Tensor) -> torch.Tensor:
        """Scatter side arrays (master frame) back to per-element local faces:
        returns [K, 6, C, q, p]; the master gets master_vals, the slave gets
        slave_vals mapped into its own local frame."""
        n = self.basis.n
        C = master_vals.shape[1]
        out = torch.zeros(self.K, 6, C, n, n, dtype=master_vals.dtype)
        out[self.m_el, self.m_sd] = master_vals
        inn = self.inner
        sv = slave_vals[inn].flatten(-2)
        idx = self.to_slave[inn].unsqueeze(1).expand(-1, C, -1)
        out[self.s_el[inn], self.s_sd[inn]] = torch.gather(sv, 2, idx).view(-1, C, n, n)
        b = self.basis
        for sd, eB, sB, typ, a, bq in self.mortar:
            sub = slave_vals[sd].flatten(-2)[:, self.to_master[sd]].view(C, n, n)  # sub-square frame
            if typ in (1, 3):
                sub = torch.einsum("ia,cqa->cqi", b.P_mortar[a], sub)
            if typ in (2, 3):
                sub = torch.einsum("jb,cbp->cjp", b.P_mortar[bq], sub)
            out[eB, sB] = out[eB, sB] + sub
        return out
