"""Pins of the oracle's geometry: Cartesian closed forms, discrete metric
identities (Eq. contravariantBasisVectorsCurl), face metric agreement and the
side orientation bookkeeping (Sec. 5.1)."""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle.basis import Basis
from oracle.mesh import MeshGeometry, apply_dir, prolong


@pytest.mark.parametrize("node_type", [0, 1])
def test_cartesian_metrics_closed_form(node_type):
    m = wl.box_mesh((3, 2, 2), Ngeo=1)
    N = 3
    geo = MeshGeometry(Basis(N, node_type), m.coords, m.conn)
    h = (m.hi - m.lo) / np.array(m.nelem)
    J = np.prod(h / 2)
    assert torch.allclose(geo.J, torch.full_like(geo.J, J), rtol=1e-13, atol=0)
    for i in range(3):
        for d in range(3):
            expect = (J / (h[i] / 2)) if i == d else 0.0  # Ja^i_d = J / (h_i/2) delta_id
            assert torch.allclose(geo.Ja[:, i, d], torch.full_like(geo.Ja[:, i, d], expect), atol=1e-13)
    # outward normals of the master sides are +-e_l and s_hat = area scale
    for sd in range(geo.nsides):
        s = int(geo.m_sd[sd])
        l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
        e = np.zeros(3); e[l] = sgn
        assert torch.allclose(geo.nvec[sd].permute(1, 2, 0), torch.tensor(e).expand(N + 1, N + 1, 3), atol=1e-13)
        assert torch.allclose(geo.sarea[sd], torch.full_like(geo.sarea[sd], J / (h[l] / 2)), rtol=1e-13)


@pytest.mark.parametrize("node_type", [0, 1])
@pytest.mark.parametrize("N", [2, 4])
def test_curved_metric_identities(node_type, N):
    m = wl.box_mesh((2, 2, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False,) * 3, reorient_seed=7)
    b = Basis(N, node_type)
    geo = MeshGeometry(b, m.coords, m.conn)
    assert geo.J.min() > 0
    for nn in range(3):
        div = sum(apply_dir(b.D, geo.Ja[:, l, nn], l) for l in range(3))
        assert div.abs().max() < 1e-12
    # x at the nodes equals the exact map up to the geometry interpolation error
    xe = torch.tensor(m.node_coords(N, node_type))
    assert (geo.x - xe).abs().max() < 0.05


@pytest.mark.parametrize("node_type", [0, 1])
def test_face_metrics_and_coordinates_agree_across_sides(node_type):
    """Both elements of a side see the same face points and opposite normals."""
    N = 4
    m = wl.box_mesh((3, 3, 2), lo=(-1,) * 3, hi=(1,) * 3, Ngeo=N, mapping="sine", periodic=(False, False, False),
                    reorient_seed=11)
    b = Basis(N, node_type)
    geo = MeshGeometry(b, m.coords, m.conn)
    xf = geo.face_values(geo.x, b.l_side)  # [K,6,3,q,p]
    XM, XS = geo.master_slave(xf)
    nt_own = []
    for s in range(6):
        l, sgn = s // 2, (-1 if s % 2 == 0 else 1)
        nt_own.append(sgn * prolong(geo.Ja[:, l], b.l_side(sgn), l))
    nt_own = torch.stack(nt_own, 1)  # [K,6,3,q,p] outward, unnormalised
    NM, NS = geo.master_slave(nt_own)
    inn = geo.inner
    assert (XM[inn] - XS[inn]).abs().max() < 1e-13
    assert (NM[inn] + NS[inn]).abs().max() < 1e-13
    assert len(geo.bnd) == 2 * (3 * 3 + 3 * 2 + 3 * 2)


def test_orientation_codes_all_used():
    m = wl.box_mesh((3, 3, 3), Ngeo=1, reorient_seed=1)
    codes = set(int(o) for o in m.conn[:, :, 2].flatten())
    assert len(codes) >= 4
    # conn symmetric: neighbour's entry points back
    for e in range(m.K):
        for s in range(6):
            nb, ns, o = m.conn[e, s]
            assert tuple(m.conn[nb, ns, :2]) == (e, s)


@pytest.mark.parametrize("node_type", [0, 1])
def test_metrics_of_a_translated_mesh(node_type):
    """The metric terms do not depend on where the mesh sits (Eq.
    contravariantBasisVectorsCurl is invariant under translation) and keep their
    closed-form values to round-off relative to the element's own size away from
    the origin: a 2^3 Cartesian box of width pi (h/2 = pi/4) placed at x = 100 has
    the same Ja and J as at the origin.  Differentiating the absolute coordinates
    directly cancels digits of magnitude 100 into sums of magnitude h/2 (errors of
    1e-12 in J and 3e-10 in Ja at N = 7); the bars below sit well above the
    round-off of the coordinates themselves (ulp(100) / (h/2) = 2e-14)."""
    N = 7
    b = Basis(N, node_type)
    h = math.pi / 2
    far = wl.box_mesh((2, 2, 2), lo=(100.0,) * 3, hi=(100.0 + math.pi,) * 3, Ngeo=1, reorient_seed=4)
    near = wl.box_mesh((2, 2, 2), lo=(0.0,) * 3, hi=(math.pi,) * 3, Ngeo=1, reorient_seed=4)
    geo = MeshGeometry(b, far.coords, far.conn)
    geo0 = MeshGeometry(b, near.coords, near.conn)
    J = (h / 2) ** 3
    assert (geo.J - J).abs().max() < 1e-13 * J
    # rotated element frames permute and flip the rows Ja^i: Ja^T Ja = (h/2)^4 I at every node
    G = torch.einsum("eadzyx,eafzyx->ezyxdf", geo.Ja, geo.Ja)
    assert (G - torch.eye(3, dtype=G.dtype) * (h / 2) ** 4).abs().max() < 1e-12 * (h / 2) ** 4
    assert (geo.Ja - geo0.Ja).abs().max() < 1e-12 * (h / 2) ** 2
    assert (geo.x - geo0.x - 100.0).abs().max() < 1e-12
