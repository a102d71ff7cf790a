"""Pins of the oracle's mortar treatment of non-conforming interfaces (Sec.
"Non-conforming meshes": interpolation of the solution from the big side to its
halves or quarters, numerical fluxes on the small sides, L2 projection back to
the big side) and of the non-conforming mesh generator."""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import equations as eq
from oracle.basis import Basis
from oracle.dgsem import DGSEM, HLLC, ROE, Params

from test_oracle_rhs import _local_to_identity_perm

GAS = eq.Gas(1.4, 0.72, 1.0 / 1600.0)
REFINE = [(1, 2, 1), (1, 1, 2), (1, 2, 2), (2, 2, 2)]


def T(a):
    return torch.tensor(a, dtype=torch.float64)


def _face_xi(s, u, v):
    l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
    other = [d for d in range(3) if d != l]
    xi = np.zeros(3)
    xi[l], xi[other[0]], xi[other[1]] = sgn, u, v
    return xi


def _orient(o, N, p, q):
    a, b = (q, p) if o & 1 else (p, q)
    return (N - a if o & 2 else a, N - b if o & 4 else b)


@pytest.mark.parametrize("refine", REFINE)
@pytest.mark.parametrize("seed", [None, 1, 4])
def test_generator_sub_faces_match_big_face(refine, seed):
    """Every small-side node, mapped by its orientation code to the sub-square of
    the big side, lies at the big side's point (eta_p' +- 1)/2 (modulo the period)."""
    N = 2
    r = wl.lobatto_points(N)
    m = wl.mortar_box_mesh(refine=refine, reorient_seed=seed, ny=1, nz=2, mapping="sine", Ngeo=2)
    assert len(m.mortars) == 4 and set(m.mortars[:, 2]) <= {1, 2, 3}
    for row in m.mortars:
        eB, sB, typ = row[:3]
        for pos in range(4):
            eS, sS, o = row[3 + 3 * pos:6 + 3 * pos]
            if eS < 0:
                assert typ != 3 and pos >= 2
                continue
            a = pos % 2 if typ == 3 else (pos if typ == 1 else 0)
            b = pos // 2 if typ == 3 else (pos if typ == 2 else 0)
            for q in range(N + 1):
                for p in range(N + 1):
                    xs = m.map_points(_face_xi(sS, r[p], r[q])[None])[eS, 0]
                    pp, qq = _orient(o, N, p, q)
                    u = (r[pp] + 2 * a - 1) / 2 if typ in (1, 3) else r[pp]
                    v = (r[qq] + 2 * b - 1) / 2 if typ in (2, 3) else r[qq]
                    xb = m.map_points(_face_xi(sB, u, v)[None])[eB, 0]
                    assert np.allclose((xs - xb + 1.0) % 2.0 - 1.0, 0.0, atol=1e-12)


@pytest.mark.parametrize("nt", [0, 1])
@pytest.mark.parametrize("N", [1, 3, 6])
def test_mortar_matrices(nt, N):
    b = Basis(N, nt)
    x, w = b.x_np, b.w_np
    rng = np.random.default_rng(N)
    c = rng.normal(size=N + 1)
    poly = lambda t: np.polynomial.polynomial.polyval(t, c)
    for a in (0, 1):
        # interpolation is exact for polynomials of degree N
        assert np.allclose(b.I_mortar[a].numpy() @ poly(x), poly((x + 2 * a - 1) / 2), atol=1e-13)
        # the projection conserves the integral: sum_i w_i (P g)_i = sum_a w_a g_a
        g = rng.normal(size=N + 1)
        assert abs(w @ (b.P_mortar[a].numpy() @ g) - w @ g) < 1e-13
    # projection of the two interpolated halves: each half's nodal flux carries
    # the half's surface element, so the sum reproduces 2 f; exact on Gauss nodes
    # (quadrature of degree 2N+1), on Gauss-Lobatto nodes for degree <= N-1
    PI = sum(b.P_mortar[a].numpy() @ b.I_mortar[a].numpy() for a in (0, 1))
    if nt == 0:
        assert np.allclose(PI, 2 * np.eye(N + 1), atol=1e-12)
    else:
        low = np.polynomial.polynomial.polyval(x, c[:N])
        assert np.allclose(PI @ low, 2 * low, atol=1e-12)
    # closed form on Gauss-Lobatto nodes at N = 1: I^0 = [[1, 0], [1/2, 1/2]]
    if nt == 1 and N == 1:
        assert np.allclose(b.I_mortar[0].numpy(), [[1, 0], [0.5, 0.5]])
        assert np.allclose(b.I_mortar[1].numpy(), [[0.5, 0.5], [0, 1]])


@pytest.mark.parametrize("refine", REFINE)
@pytest.mark.parametrize("nt", [0, 1])
def test_interpolated_states_match_small_faces_for_linear_fields(refine, nt):
    """For a linear field (exact in every element) the big side's solution
    interpolated to a small side equals the small element's own face values."""
    N = 3
    m = wl.mortar_box_mesh(refine=refine, reorient_seed=2, ny=1, nz=2, periodic=(False, True, True))
    dg = DGSEM(Params(N=N, node_type=nt), m.coords, m.conn, m.mortars)
    x = T(m.node_coords(N, nt))
    f = (1.0 + 0.3 * x[:, 0] - 0.2 * x[:, 1] + 0.7 * x[:, 2]).unsqueeze(1)  # [K,1,n,n,n]
    faces = dg.geo.face_values(f, dg.b.l_side)
    M, S = dg.geo.master_slave(faces)
    v = dg.geo.virt
    assert len(v) > 0
    assert torch.allclose(M[v], S[v], atol=1e-13, rtol=0)


@pytest.mark.parametrize("refine", REFINE)
def test_projection_inverts_interpolation_gauss(refine):
    """Gauss nodes: projecting the interpolated big-side values back returns them
    times the number of sub-faces (each small side's value carries its share of
    the surface element)."""
    N = 4
    m = wl.mortar_box_mesh(refine=refine, reorient_seed=7, ny=1, nz=2)
    dg = DGSEM(Params(N=N, node_type=0), m.coords, m.conn, m.mortars)
    rng = np.random.default_rng(0)
    faces = T(rng.normal(size=(m.K, 6, 2, N + 1, N + 1)))
    _, S = dg.geo.master_slave(faces)
    back = dg.geo.to_elements(torch.zeros_like(S), S)
    for row in m.mortars:
        eB, sB, typ = int(row[0]), int(row[1]), int(row[2])
        nsub = 4 if typ == 3 else 2
        assert torch.allclose(back[eB, sB], nsub * faces[eB, sB], atol=1e-12)


@pytest.mark.parametrize("refine", REFINE)
@pytest.mark.parametrize("nt,mapping", [(0, "cartesian"), (0, "sine"), (1, "sine")])
def test_mortar_freestream(refine, nt, mapping):
    N = 3
    m = wl.mortar_box_mesh(refine=refine, reorient_seed=3, ny=1, nz=2, mapping=mapping,
                           Ngeo=N if mapping == "sine" else 1)
    dg = DGSEM(Params(N=N, node_type=nt, riemann=HLLC), m.coords, m.conn, m.mortars)
    Ut = dg.rhs(T(wl.freestream(m.node_coords(N, nt))))
    assert float(Ut.abs().max()) < 1e-12


@pytest.mark.parametrize("riemann", [ROE, HLLC])
@pytest.mark.parametrize("nt", [0, 1])
def test_mortar_conservation(riemann, nt):
    N = 3
    m = wl.mortar_box_mesh(refine=(1, 2, 2), reorient_seed=5, ny=2, nz=1, mapping="sine", Ngeo=3)
    dg = DGSEM(Params(N=N, node_type=nt, riemann=riemann), m.coords, m.conn, m.mortars)
    Ut = dg.rhs(T(wl.perturbed(np.pi * m.node_coords(N, nt), seed=4)))
    wJ = dg.quad_weights().unsqueeze(1)
    tot = (wJ * Ut).sum(dim=(0, 2, 3, 4))
    scale = (wJ * Ut.abs()).sum(dim=(0, 2, 3, 4))
    assert float((tot.abs() / scale).max()) < 1e-13


@pytest.mark.parametrize("nt", [0, 1])
def test_mortar_reorientation_invariance(nt):
    """Element frames (and hence side orientations and mortar positions in the
    big side's frame) must not change the result."""
    N = 3
    res = []
    for seed in (None, 11):
        m = wl.mortar_box_mesh(refine=(2, 2, 2), reorient_seed=seed, ny=1, nz=1)
        dg = DGSEM(Params(N=N, node_type=nt, riemann=HLLC), m.coords, m.conn, m.mortars)
        R = dg.rhs(T(wl.perturbed(np.pi * m.node_coords(N, nt), seed=3)))
        if seed is not None:
            perm = torch.tensor(_local_to_identity_perm(m, N))
            R = torch.gather(R.flatten(2), 2, perm.unsqueeze(1).expand(-1, 5, -1)).view_as(R)
        res.append(R)
    assert float((res[0] - res[1]).abs().max()) < 1e-12 * float(res[0].abs().max())


def _mms_error(N, nel, nt, refine):
    """Manufactured solution on the curved periodic two-block mesh with cubic
    elements of width 1/nel (left block) and 1/(2 nel) (right block, refine 2)."""
    m = wl.mortar_box_mesh(refine=refine, ny=2 * nel, nz=2 * nel, nx=nel, mapping="sine", Ngeo=N)
    dg = DGSEM(Params(N=N, node_type=nt, riemann=HLLC, source=True), m.coords, m.conn, m.mortars)
    x = dg.geo.x.movedim(1, -1)
    U0 = eq.exact_state(eq.EXACT_MANUFACTURED, x, 0.0, GAS).movedim(-1, 1).contiguous()
    t_end = 0.05
    nsteps = int(math.ceil(t_end / (0.05 / nel / (N + 1))))
    U = dg.run(U0, nsteps, t_end / nsteps)
    Ue = eq.exact_state(eq.EXACT_MANUFACTURED, x, t_end, GAS).movedim(-1, 1)
    return math.sqrt(float((dg.quad_weights() * (U[:, 0] - Ue[:, 0]) ** 2).sum()))


@pytest.mark.parametrize("nt", [0, 1])
def test_mortar_manufactured_convergence(nt):
    """Type-3 mortars at both interfaces of a curved periodic mesh (N = 2,
    nel = 1, 2, 3): the error is below that of the same mesh without the
    refined half at every level, and the observed order matches the conforming
    mesh's (pre-asymptotic at these sizes: about 2.4 for Gauss and 2.1 for
    Gauss-Lobatto nodes on both meshes)."""
    N = 2
    em = [_mms_error(N, nel, nt, (2, 2, 2)) for nel in (1, 2, 3)]
    ec = [_mms_error(N, nel, nt, (1, 1, 1)) for nel in (1, 2, 3)]
    order = lambda e: math.log(e[1] / e[2]) / math.log(1.5)
    assert all(a < b for a, b in zip(em, ec)), (em, ec)
    assert em[0] > em[1] > em[2] and order(em) > N - 0.5, (em, order(em))
    assert abs(order(em) - order(ec)) < 0.15, (order(em), order(ec))
