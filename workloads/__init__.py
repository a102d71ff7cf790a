"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *generates inputs*: hexahedral box meshes (node coordinates at
Gauss-Lobatto geometry points plus face connectivity with orientation codes) and
nodal initial states sampled from closed-form fields.  It contains none of the
DGSEM arithmetic (no differentiation matrices, metrics, fluxes or time
integration); the two implementations that consume these inputs each do that
themselves.

Conventions (they define the mesh interface, Sec. 3.1 and Sec. 5.1 of the paper):

* Element-local volume indices (i, j, k) run along (xi1, xi2, xi3); arrays are
  stored ``[..., k, j, i]`` with i fastest.
* Local sides: 0: xi1=-1, 1: xi1=+1, 2: xi2=-1, 3: xi2=+1, 4: xi3=-1, 5: xi3=+1.
* Side-local face coordinates (p, q): the two remaining volume indices in
  increasing direction order, i.e. (j,k) on xi1 faces, (i,k) on xi2 faces and
  (i,j) on xi3 faces.  Face arrays are stored ``[..., q, p]``.
* Orientation code o in 0..7 maps a face node (p, q) of one element to the node
  (p', q') of the neighbour's side-local system: (a, b) = (q, p) if o & 1 else
  (p, q); p' = N - a if o & 2 else a; q' = N - b if o & 4 else b.
* conn[e, s] = (neighbour element, neighbour local side, o) or (-1 - bc_id, -1, 0)
  on a boundary.
* Non-conforming (mortar) interfaces, Sec. 4 "Non-conforming meshes": a big side
  is cut at the middle of its reference square into two halves along p (type 1),
  along q (type 2) or into four quarters (type 3).  Sides on such an interface
  have conn[e, s] = (MORTAR, m, pos), pos = -1 for the big side, and row m of
  ``mortars`` is (big element, big local side, type, then for pos = 0..3 the
  small element, its local side and the orientation code o that maps its
  side-local (p, q) to the node (p', q') of the sub-square in the big side's
  frame, rescaled to the full index range; -1 where unused).  Position pos is
  a (type 1), b (type 2) or a + 2 b (type 3), with a = 0 / 1 for the lower /
  upper half along p and b likewise along q.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

# ----------------------------------------------------------------------------
# node sets used only to *sample* geometry and initial states (numpy library)
# ----------------------------------------------------------------------------


def lobatto_points(N: int) -> np.ndarray:
    """Gauss-Lobatto points on [-1, 1] (numpy root finder on P'_N)."""
    if N == 0:
        return np.array([0.0])
    from numpy.polynomial import legendre as L

    c = np.zeros(N + 1)
    c[N] = 1.0
    inner = np.sort(np.real(L.legroots(L.legder(c)))) if N > 1 else np.array([])
    return np.concatenate([[-1.0], inner, [1.0]])


def gauss_points(N: int) -> np.ndarray:
    from numpy.polynomial import legendre as L

    return L.leggauss(N + 1)[0]


def solution_points(N: int, node_type: int) -> np.ndarray:
    """node_type 0: Legendre-Gauss, 1: Legendre-Gauss-Lobatto."""
    return gauss_points(N) if node_type == 0 else lobatto_points(N)


# ----------------------------------------------------------------------------
# element frames: the 24 proper rotations of the cube (signed permutations)
# ----------------------------------------------------------------------------


def cube_rotations() -> list[np.ndarray]:
    rots = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                R[r, perm[r]] = signs[r]
            if round(np.linalg.det(R)) == 1:
                rots.append(R)
    return rots


def orientation_code(pmap) -> int:
    """Return o such that the map (p, q) -> (p', q') on an N=1 face matches pmap."""
    for o in range(8):
        ok = True
        for p, q in ((0, 0), (1, 0), (0, 1), (1, 1)):
            a, b = (q, p) if o & 1 else (p, q)
            pp = 1 - a if o & 2 else a
            qq = 1 - b if o & 4 else b
            if (pp, qq) != pmap[(p, q)]:
                ok = False
                break
        if ok:
            return o
    raise ValueError("face maps are not a dihedral transform")


def _face_corner_xi(s: int, p: int, q: int) -> np.ndarray:
    """Local reference coordinate (+-1 components) of face corner (p, q) of side s."""
    l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
    other = [d for d in range(3) if d != l]
    xi = np.zeros(3)
    xi[l] = sgn
    xi[other[0]] = -1 + 2 * p
    xi[other[1]] = -1 + 2 * q
    return xi


@dataclass
class BoxMesh:
    """A structured box of hexahedra presented as an unstructured mesh."""

    nelem: tuple  # (nx, ny, nz)
    Ngeo: int
    coords: np.ndarray  # [K, Ngeo+1, Ngeo+1, Ngeo+1, 3] at LGL points, [e, k, j, i, xyz]
    conn: np.ndarray  # [K, 6, 3] int32
    lattice: np.ndarray  # [K, 3] integer lattice position of each element
    frames: np.ndarray  # [K, 3, 3] local->global signed permutation R (eta = R xi)
    lo: np.ndarray
    hi: np.ndarray
    mapping: str

    @property
    def K(self) -> int:
        return self.lattice.shape[0]

    def map_points(self, xi_local: np.ndarray) -> np.ndarray:
        """Physical coordinates of element-local reference points.

        xi_local: [..., 3] in [-1,1]^3 (same for every element).  Returns
        [K, ..., 3] using the exact (analytic) mapping, not an interpolant.
        """
        h = (self.hi - self.lo) / np.array(self.nelem)
        eta = np.einsum("kab,...b->k...a", self.frames.astype(float), xi_local)
        shp = (self.K,) + (1,) * (xi_local.ndim - 1) + (3,)
        lat = self.lattice.reshape(shp).astype(float)
        x = self.lo + (lat + (eta + 1.0) / 2.0) * h
        return _apply_mapping(x, self.mapping, self.lo, self.hi)

    def node_coords(self, N: int, node_type: int) -> np.ndarray:
        """Exact physical coordinates at the solution nodes, [K, 3, n, n, n]."""
        r = solution_points(N, node_type)
        kk, jj, ii = np.meshgrid(r, r, r, indexing="ij")
        xi = np.stack([ii, jj, kk], axis=-1)  # [k, j, i, 3]
        x = self.map_points(xi)  # [K, k, j, i, 3]
        return np.ascontiguousarray(np.moveaxis(x, -1, 1))


def _apply_mapping(x: np.ndarray, mapping: str, lo, hi) -> np.ndarray:
    if mapping == "cartesian":
        return x
    if mapping == "sine":
        # x_i = xi_i + 0.1 * prod_j sin(pi xi_j), xi the global coordinate in [-1,1]^3
        xi = 2.0 * (x - lo) / (hi - lo) - 1.0
        bump = 0.1 * np.prod(np.sin(np.pi * xi), axis=-1, keepdims=True)
        return lo + (xi + bump + 1.0) * (hi - lo) / 2.0
    raise ValueError(mapping)


def box_mesh(nelem=(4, 4, 4), lo=(0.0, 0.0, 0.0), hi=(2 * math.pi,) * 3, Ngeo: int = 1,
             periodic=(True, True, True), mapping: str = "cartesian", reorient_seed=None,
             bc_ids=None) -> BoxMesh:
    """Box of nx*ny*nz hexahedra.

    reorient_seed: if not None, every element gets a random proper rotation of its
    local frame (exercises side orientations).  bc_ids: 6 boundary ids for the
    box faces (-x,+x,-y,+y,-z,+z); default 0 everywhere.
    """
    nx, ny, nz = nelem
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    bc_ids = bc_ids if bc_ids is not None else [0] * 6
    lattice = np.array([(a, b, c) for c in range(nz) for b in range(ny) for a in range(nx)], dtype=np.int64)
    K = len(lattice)
    rots = cube_rotations()
    if reorient_seed is None:
        frames = np.tile(np.eye(3, dtype=np.int64), (K, 1, 1))
    else:
        rng = np.random.default_rng(reorient_seed)
        frames = np.stack([rots[rng.integers(len(rots))] for _ in range(K)])
    index = {tuple(p): e for e, p in enumerate(lattice)}
    dims = np.array(nelem)
    conn = np.zeros((K, 6, 3), dtype=np.int32)
    for e in range(K):
        R = frames[e]
        for s in range(6):
            l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
            step = R[:, l] * sgn  # outward lattice direction
            nb_pos = lattice[e] + step
            gdir = int(np.nonzero(step)[0][0])
            if nb_pos[gdir] < 0 or nb_pos[gdir] >= dims[gdir]:
                if not periodic[gdir]:
                    face = 2 * gdir + (0 if step[gdir] < 0 else 1)
                    conn[e, s] = (-1 - bc_ids[face], -1, 0)
                    continue
            nb_wrapped = nb_pos % dims
            nb = index[tuple(nb_wrapped)]
            Rn = frames[nb]
            # neighbour side: outward direction opposite to ours
            sn = None
            for t in range(6):
                ln, sgnn = t // 2, (-1 if t % 2 == 0 else 1)
                if np.array_equal(Rn[:, ln] * sgnn, -step):
                    sn = t
                    break
            # corner correspondence in lattice units (unwrapped neighbour box)
            pmap = {}
            for p, q in ((0, 0), (1, 0), (0, 1), (1, 1)):
                xi = _face_corner_xi(s, p, q)
                Lpt = lattice[e] + (R @ xi + 1) / 2.0
                rel = Lpt - nb_pos
                xin = Rn.T @ (2 * rel - 1)
                ln = sn // 2
                other = [d for d in range(3) if d != ln]
                pmap[(p, q)] = (int(round((xin[other[0]] + 1) / 2)), int(round((xin[other[1]] + 1) / 2)))
            conn[e, s] = (nb, sn, orientation_code(pmap))
    # geometry at Ngeo LGL points in each element's local frame
    r = lobatto_points(Ngeo)
    kk, jj, ii = np.meshgrid(r, r, r, indexing="ij")
    xi = np.stack([ii, jj, kk], axis=-1)
    mesh = BoxMesh(nelem=tuple(nelem), Ngeo=Ngeo, coords=None, conn=conn, lattice=lattice, frames=frames,
                   lo=lo, hi=hi, mapping=mapping)
    mesh.coords = np.ascontiguousarray(mesh.map_points(xi))
    return mesh


MORTAR = -(1 << 30)  # conn neighbour value of a side on a mortar interface


@dataclass
class NCMesh:
    """Hexahedra as axis-aligned boxes of a global integer grid (not necessarily
    conforming), presented as an unstructured mesh with mortar interfaces."""

    box_lo: np.ndarray  # [K, 3] lower corner in grid units
    box_size: np.ndarray  # [K, 3] extent in grid units
    dims: np.ndarray  # [3] domain extent in grid units
    frames: np.ndarray  # [K, 3, 3] local->global signed permutation
    Ngeo: int
    coords: np.ndarray
    conn: np.ndarray
    mortars: np.ndarray  # [M, 15] int32
    lo: np.ndarray
    hi: np.ndarray
    mapping: str

    @property
    def K(self) -> int:
        return self.box_lo.shape[0]

    def map_points(self, xi_local: np.ndarray) -> np.ndarray:
        eta = np.einsum("kab,...b->k...a", self.frames.astype(float), xi_local)
        shp = (self.K,) + (1,) * (xi_local.ndim - 1) + (3,)
        L = self.box_lo.reshape(shp).astype(float)
        Sz = self.box_size.reshape(shp).astype(float)
        x = self.lo + (L + (eta + 1.0) / 2.0 * Sz) * (self.hi - self.lo) / self.dims
        return _apply_mapping(x, self.mapping, self.lo, self.hi)

    def node_coords(self, N: int, node_type: int) -> np.ndarray:
        r = solution_points(N, node_type)
        kk, jj, ii = np.meshgrid(r, r, r, indexing="ij")
        x = self.map_points(np.stack([ii, jj, kk], axis=-1))
        return np.ascontiguousarray(np.moveaxis(x, -1, 1))


def _connect_boxes(box_lo, box_size, dims, frames, periodic, bc_ids):
    """Face connectivity of a set of boxes: conforming neighbours, boundaries and
    2:1 mortar interfaces (found geometrically, with periodic wrap)."""
    K = box_lo.shape[0]
    faces = {}  # (axis, plane) -> list of (e, s, dirsign, rect)
    info = {}
    for e in range(K):
        R = frames[e]
        for s in range(6):
            l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
            step = R[:, l] * sgn
            g = int(np.nonzero(step)[0][0])
            ds = int(step[g])
            c = int(box_lo[e, g] + (box_size[e, g] if ds > 0 else 0))
            o1, o2 = [d for d in range(3) if d != g]
            rect = (int(box_lo[e, o1]), int(box_lo[e, o1] + box_size[e, o1]),
                    int(box_lo[e, o2]), int(box_lo[e, o2] + box_size[e, o2]))
            bnd = (c == 0 or c == dims[g]) and not periodic[g]
            cm = c % dims[g] if periodic[g] else c
            info[(e, s)] = (g, ds, cm, rect, bnd, c)
            faces.setdefault((g, cm), []).append((e, s, ds, rect))

    def corners(e, s):
        """In-plane grid coordinates of the face corners (p, q) in {0,1}^2."""
        g = info[(e, s)][0]
        o1, o2 = [d for d in range(3) if d != g]
        out = {}
        for p, q in ((0, 0), (1, 0), (0, 1), (1, 1)):
            xi = _face_corner_xi(s, p, q)
            X = box_lo[e] + (frames[e] @ xi + 1) / 2.0 * box_size[e]
            out[(p, q)] = np.array([X[o1], X[o2]])
        return out

    conn = np.zeros((K, 6, 3), dtype=np.int32)
    mortars = []
    for e in range(K):
        for s in range(6):
            g, ds, cm, rect, bnd, c = info[(e, s)]
            if bnd:
                face = 2 * g + (0 if ds < 0 else 1)
                conn[e, s] = (-1 - bc_ids[face], -1, 0)
                continue
            cands = [(e2, s2, r2) for (e2, s2, ds2, r2) in faces[(g, cm)]
                     if ds2 == -ds and min(rect[1], r2[1]) > max(rect[0], r2[0])
                     and min(rect[3], r2[3]) > max(rect[2], r2[2])]
            area = lambda r: (r[1] - r[0]) * (r[3] - r[2])
            if len(cands) == 1 and cands[0][2] == rect:
                e2, s2, _ = cands[0]
                mine, theirs = corners(e, s), corners(e2, s2)
                pmap = {pq: next(k for k, v in theirs.items() if np.allclose(v, x)) for pq, x in mine.items()}
                conn[e, s] = (e2, s2, orientation_code(pmap))
            elif len(cands) == 1 and area(cands[0][2]) > area(rect):
                continue  # small side of a mortar: filled from the big side
            else:
                if sum(area(r) for _, _, r in cands) != area(rect) or len(cands) not in (2, 4):
                    raise ValueError("unsupported non-conforming interface")
                big = corners(e, s)
                A = big[(0, 0)]
                up, uq = big[(1, 0)] - A, big[(0, 1)] - A
                row = [e, s, 0] + [-1] * 12
                m = len(mortars)
                for e2, s2, r2 in cands:
                    sm = corners(e2, s2)
                    nrm = lambda X: (float((X - A) @ up / (up @ up)), float((X - A) @ uq / (uq @ uq)))
                    st = [nrm(x) for x in sm.values()]
                    dp = max(a for a, _ in st) - min(a for a, _ in st)
                    dq = max(b for _, b in st) - min(b for _, b in st)
                    typ = {(0.5, 1.0): 1, (1.0, 0.5): 2, (0.5, 0.5): 3}[(round(dp, 6), round(dq, 6))]
                    ctr = (sum(a for a, _ in st) / 4, sum(b for _, b in st) / 4)
                    a = int(ctr[0] > 0.5) if dp < 1 else 0
                    b = int(ctr[1] > 0.5) if dq < 1 else 0
                    pos = {1: a, 2: b, 3: a + 2 * b}[typ]
                    pmap = {}
                    for pq, X in sm.items():
                        s1, s2v = nrm(X)
                        pp = int(round(2 * s1 - a)) if dp < 1 else int(round(s1))
                        qq = int(round(2 * s2v - b)) if dq < 1 else int(round(s2v))
                        pmap[pq] = (pp, qq)
                    row[2] = typ
                    row[3 + 3 * pos:6 + 3 * pos] = [e2, s2, orientation_code(pmap)]
                    conn[e2, s2] = (MORTAR, m, pos)
                conn[e, s] = (MORTAR, m, -1)
                mortars.append(row)
    return conn, np.array(mortars, dtype=np.int32).reshape(-1, 15)


def mortar_box_mesh(ny: int = 2, nz: int = 2, nx: int = 1, refine=(1, 2, 2), lo=(-1.0,) * 3, hi=(1.0,) * 3,
                    Ngeo: int = 1, periodic=(True, True, True), mapping: str = "cartesian",
                    reorient_seed=None, bc_ids=None) -> NCMesh:
    """Two blocks of equal width in x: the left one of nx * ny * nz elements, the
    right one refined by refine = (rx, ry, rz) in {1, 2}^3 (ry * rz > 1).  The
    interface at the middle of the box (and, with periodic x, the one at its
    ends) is non-conforming: type 3 mortars for ry = rz = 2, halves otherwise.
    With the "sine" mapping on [-1, 1]^3 both interfaces lie on planes where the
    bump vanishes, so big and small faces are the same flat patches."""
    rx, ry, rz = refine
    cl, fl = [], []
    for c in range(nz):
        for b in range(ny):
            for a in range(nx):
                cl.append(((2 * a, 2 * b, 2 * c), (2, 2, 2)))
    sx, sy, sz = 2 // rx, 2 // ry, 2 // rz
    for c in range(nz * rz):
        for b in range(ny * ry):
            for a in range(nx * rx):
                fl.append(((2 * nx + sx * a, sy * b, sz * c), (sx, sy, sz)))
    boxes = cl + fl
    box_lo = np.array([b[0] for b in boxes], dtype=np.int64)
    box_size = np.array([b[1] for b in boxes], dtype=np.int64)
    dims = np.array([4 * nx, 2 * ny, 2 * nz], dtype=np.int64)
    K = len(boxes)
    rots = cube_rotations()
    if reorient_seed is None:
        frames = np.tile(np.eye(3, dtype=np.int64), (K, 1, 1))
    else:
        rng = np.random.default_rng(reorient_seed)
        frames = np.stack([rots[rng.integers(len(rots))] for _ in range(K)])
    conn, mortars = _connect_boxes(box_lo, box_size, dims, frames, periodic, bc_ids if bc_ids else [0] * 6)
    r = lobatto_points(Ngeo)
    kk, jj, ii = np.meshgrid(r, r, r, indexing="ij")
    mesh = NCMesh(box_lo=box_lo, box_size=box_size, dims=dims, frames=frames, Ngeo=Ngeo, coords=None, conn=conn,
                  mortars=mortars, lo=np.asarray(lo, float), hi=np.asarray(hi, float), mapping=mapping)
    mesh.coords = np.ascontiguousarray(mesh.map_points(np.stack([ii, jj, kk], axis=-1)))
    return mesh


def reorder_to_local(field_global_frame_fn, mesh: BoxMesh, N: int, node_type: int):
    """Evaluate a pointwise field at each element's own node ordering."""
    x = mesh.node_coords(N, node_type)
    return field_global_frame_fn(x)


# ----------------------------------------------------------------------------
# initial states (nodal samples of closed-form fields); U layout [K, 5, n, n, n]
# ----------------------------------------------------------------------------


def prim_to_cons_np(rho, u, v, w, p, gamma):
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E], axis=1)


def taylor_green(x: np.ndarray, Ma: float = 0.1, gamma: float = 1.4, const_pressure: bool = False) -> np.ndarray:
    """Taylor-Green vortex, V0 = L = rho0 = 1, p0 = 1/(gamma Ma^2)."""
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p0 = 1.0 / (gamma * Ma * Ma)
    if const_pressure:
        p = np.full_like(u, p0)
    else:
        p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    rho = np.ones_like(u)
    return prim_to_cons_np(rho, u, v, w, p, gamma)


def freestream(x: np.ndarray, rho=1.0, vel=(0.3, 0.2, 0.1), p=None, gamma: float = 1.4) -> np.ndarray:
    p = 1.0 / gamma if p is None else p
    one = np.ones_like(x[:, 0])
    return prim_to_cons_np(rho * one, vel[0] * one, vel[1] * one, vel[2] * one, p * one, gamma)


def manufactured(x: np.ndarray, t: float = 0.0) -> np.ndarray:
    """rho = 2 + 0.1 sin(pi (x+y+z-2t)), m = (rho, rho, rho), rho E = rho^2."""
    rho = 2.0 + 0.1 * np.sin(np.pi * (x[:, 0] + x[:, 1] + x[:, 2] - 2.0 * t))
    return np.stack([rho, rho, rho, rho, rho * rho], axis=1)


def perturbed(x: np.ndarray, seed: int, amp: float = 0.05, Ma: float = 0.3, gamma: float = 1.4) -> np.ndarray:
    """Smooth random state: a few seeded Fourier modes on top of a uniform flow.

    Used where a generic (non-symmetric) state is wanted; periodic on [0, 2 pi]^3
    for integer wave numbers.
    """
    rng = np.random.default_rng(seed)
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]

    def field():
        f = np.zeros_like(X)
        for _ in range(4):
            kx, ky, kz = rng.integers(-2, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            a = rng.normal()
            f = f + a * np.sin(kx * X + ky * Y + kz * Z + ph)
        return f

    rho = 1.0 + amp * field()
    u = 0.3 + 3 * amp * field()
    v = -0.2 + 3 * amp * field()
    w = 0.1 + 3 * amp * field()
    p = 1.0 / (gamma * Ma * Ma) * (1.0 + amp * field())
    return prim_to_cons_np(rho, u, v, w, p, gamma)


def random_directions(shape, count: int, seed0: int = 1910, norm: str = "l2") -> list[np.ndarray]:
    """Seeded random directions with N(0,1) entries (seed seed0 + i), scaled to
    unit L2 norm (norm="l2") or to unit RMS per entry (norm="rms", i.e. left as
    drawn up to the sample RMS)."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        v = rng.normal(size=shape)
        scale = np.linalg.norm(v) if norm == "l2" else np.sqrt(np.mean(v * v))
        out.append(v / scale)
    return out
