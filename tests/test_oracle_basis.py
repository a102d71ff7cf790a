"""Pins of the oracle's 1-D operators against closed forms and library routines
(nodes/weights, D, Lagrange values, D_hat / l_hat identities; Sec. 3.1)."""
import math
import os

import numpy as np
import pytest

from oracle.basis import Basis, diff_matrix, gauss_nodes, lagrange_at, lobatto_nodes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_closed_form_nodes_weights():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "quadrature_closed_forms.txt")) if l.strip() and l[0] != "#"]
    for fam, N, xs, ws in rows:
        N = int(N)
        x, w = (gauss_nodes(N) if fam == "LG" else lobatto_nodes(N))
        xv, wv = eval(xs, {"math": math}), eval(ws, {"math": math})
        i = int(np.argmin(np.abs(x - xv)))
        assert abs(x[i] - xv) < 1e-15 and abs(w[i] - wv) < 1e-15, (fam, N, xs)


@pytest.mark.parametrize("N", range(0, 12))
def test_gauss_matches_numpy(N):
    x, w = gauss_nodes(N)
    xr, wr = np.polynomial.legendre.leggauss(N + 1)
    assert np.allclose(x, xr, atol=1e-14, rtol=0) and np.allclose(w, wr, atol=1e-14, rtol=0)


@pytest.mark.parametrize("N", range(1, 12))
@pytest.mark.parametrize("node_type", [0, 1])
def test_quadrature_exactness_degree(N, node_type):
    """LG exact to degree 2N+1, LGL to 2N-1 (Sec. 3.1, mass matrix discussion)."""
    x, w = gauss_nodes(N) if node_type == 0 else lobatto_nodes(N)
    top = 2 * N + 1 if node_type == 0 else 2 * N - 1
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(top + 1):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-13
    k = top + 1  # first degree that is not integrated exactly (even)
    assert abs(np.sum(w * x ** k) - 2.0 / (k + 1)) > 1e-9
    assert np.allclose(x, -x[::-1], atol=1e-15) and np.allclose(w, w[::-1], atol=1e-15)


@pytest.mark.parametrize("N", range(1, 10))
@pytest.mark.parametrize("node_type", [0, 1])
def test_D_exact_on_polynomials(N, node_type):
    x, _ = gauss_nodes(N) if node_type == 0 else lobatto_nodes(N)
    D = diff_matrix(x)
    assert np.max(np.abs(D @ np.ones_like(x))) < 1e-12
    for m in range(1, N + 1):
        assert np.max(np.abs(D @ x ** m - m * x ** (m - 1))) < 1e-11 * max(1, m)


@pytest.mark.parametrize("N", range(1, 10))
@pytest.mark.parametrize("node_type", [0, 1])
def test_lagrange_endpoints(N, node_type):
    x, _ = gauss_nodes(N) if node_type == 0 else lobatto_nodes(N)
    for xi in (-1.0, 1.0, 0.3):
        l = lagrange_at(x, xi)
        for m in range(N + 1):
            assert abs(np.dot(l, x ** m) - xi ** m) < 1e-12
    if node_type == 1:
        assert np.allclose(lagrange_at(x, -1.0), np.eye(N + 1)[0]) and np.allclose(lagrange_at(x, 1.0), np.eye(N + 1)[-1])


@pytest.mark.parametrize("N", range(1, 10))
@pytest.mark.parametrize("node_type", [0, 1])
def test_constant_flux_identity(N, node_type):
    """sum_a Dhat_ia + lhat_i(1) - lhat_i(-1) = 0: a constant flux has zero
    divergence (follows from Eq. semiDiscrete).  The variant printed in the paper,
    -(w_i/w_j) D_ji, violates it for N >= 2 (reading of Dhat)."""
    b = Basis(N, node_type)
    Dh = b.Dhat.numpy()
    res = Dh.sum(1) + b.lhat_plus.numpy() - b.lhat_minus.numpy()
    assert np.max(np.abs(res)) < 1e-12
    if N >= 2:
        w, D = b.w_np, b.D_np
        printed = -(w[:, None] / w[None, :]) * D.T
        res2 = printed.sum(1) + b.lhat_plus.numpy() - b.lhat_minus.numpy()
        assert np.max(np.abs(res2)) > 1e-3


@pytest.mark.parametrize("N", range(1, 10))
@pytest.mark.parametrize("node_type", [0, 1])
def test_weak_equals_strong_1d(N, node_type):
    """For a polynomial v of degree <= N the weak operator
    Dhat v + lhat(1) v(1) - lhat(-1) v(-1) equals the strong derivative D v
    (summation by parts; Sec. 3.1 'Strong formulation')."""
    b = Basis(N, node_type)
    x = b.x_np
    rng = np.random.default_rng(N)
    c = rng.normal(size=N + 1)
    v = np.polyval(c, x)
    v1, vm1 = np.polyval(c, 1.0), np.polyval(c, -1.0)
    weak = b.Dhat.numpy() @ v + b.lhat_plus.numpy() * v1 - b.lhat_minus.numpy() * vm1
    assert np.max(np.abs(weak - b.D_np @ v)) < 1e-10
