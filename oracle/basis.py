"""One-dimensional DGSEM building blocks (oracle; test infrastructure only).

* Legendre-Gauss (LG) and Legendre-Gauss-Lobatto (LGL) nodes and weights
  (Sec. 3.1, "The nodal points r_i are taken from either LG or LGL quadrature").
  Textbook construction: Newton iteration on P_{N+1} (LG) or on P'_N (LGL) from
  Chebyshev starting guesses; w = 2/((1-x^2) P'_{N+1}(x)^2) (LG),
  w = 2/(N(N+1) P_N(x)^2) (LGL).
* Lagrange polynomials l_j by their product definition (Sec. 3.1).
* Differentiation matrix D_rs = l_s'(xi_r) (Eq. discVolInt and the definition
  just before it), evaluated with the barycentric formula (Berrut & Trefethen,
  "Barycentric Lagrange interpolation", SIAM Review 2004): off-diagonal
  D_rs = (w_s/w_r)/(x_r - x_s), diagonal = -sum of the row's off-diagonals.
* D_hat and l_hat (the precomputed operators after Eq. semiDiscrete).  Reading:
  the paper prints D_hat_ij = -(w_i/w_j) D_ji; redoing the quadrature of the
  volume term (the derivation leading to Eq. discVolInt, divided by the mass
  matrix of Eq. discTemp) gives D_hat_ij = -(w_j/w_i) D_ji, the only version
  that differentiates a constant flux to zero together with l_hat.  The tests
  pin that identity.
* Mortar interpolation and projection matrices (Sec. "Non-conforming meshes").
"""
from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.float64


def legendre(N: int, x: np.ndarray):
    """P_N(x) and P_N'(x) by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    if N == 0:
        return np.ones_like(x), np.zeros_like(x)
    p0, p1 = np.ones_like(x), x.copy()
    d0, d1 = np.zeros_like(x), np.ones_like(x)
    for k in range(2, N + 1):
        p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        d2 = d0 + (2 * k - 1) * p1
        p0, p1, d0, d1 = p1, p2, d1, d2
    return p1, d1


def gauss_nodes(N: int):
    """N+1 Legendre-Gauss nodes and weights on [-1, 1]."""
    n = N + 1
    x = -np.cos(np.pi * (2 * np.arange(n) + 1) / (2 * n))  # Chebyshev-Gauss guesses, ascending
    for _ in range(100):
        p, dp = legendre(n, x)
        dx = p / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    _, dp = legendre(n, x)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def lobatto_nodes(N: int):
    """N+1 Legendre-Gauss-Lobatto nodes and weights on [-1, 1] (N >= 1)."""
    if N < 1:
        raise ValueError("LGL needs N >= 1")
    x = -np.cos(np.pi * np.arange(N + 1) / N)  # Chebyshev-Gauss-Lobatto guesses
    inner = x[1:-1].copy()
    for _ in range(100):
        p, dp = legendre(N, inner)
        # P_N'' from Legendre's equation (1-x^2)P'' - 2xP' + N(N+1)P = 0
        ddp = (2 * inner * dp - N * (N + 1) * p) / (1 - inner * inner)
        dx = dp / ddp
        inner = inner - dx
        if inner.size == 0 or np.max(np.abs(dx)) < 1e-16:
            break
    x = np.concatenate([[-1.0], inner, [1.0]])
    p, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * p * p)
    return x, w


def nodes_weights(N: int, node_type: int):
    """node_type 0: LG, 1: LGL."""
    return gauss_nodes(N) if node_type == 0 else lobatto_nodes(N)


def lagrange_at(x: np.ndarray, xi: float) -> np.ndarray:
    """Vector l_j(xi), j = 0..N, from the product definition."""
    n = len(x)
    out = np.ones(n)
    for j in range(n):
        for i in range(n):
            if i != j:
                out[j] *= (xi - x[i]) / (x[j] - x[i])
    return out


def lagrange_matrix(x_from: np.ndarray, x_to: np.ndarray) -> np.ndarray:
    """V[r, j] = l_j(x_to[r]) for the Lagrange basis on x_from (interpolation)."""
    return np.stack([lagrange_at(x_from, t) for t in x_to])


def diff_matrix(x: np.ndarray) -> np.ndarray:
    """D[r, s] = l_s'(x_r) (barycentric form)."""
    n = len(x)
    wb = np.array([1.0 / np.prod([x[j] - x[k] for k in range(n) if k != j]) for j in range(n)])
    D = np.zeros((n, n))
    for r in range(n):
        for s in range(n):
            if r != s:
                D[r, s] = (wb[s] / wb[r]) / (x[r] - x[s])
        D[r, r] = -np.sum(D[r, :])
    return D


class Basis:
    """All 1-D operators for polynomial degree N on LG (0) or LGL (1) nodes."""

    def __init__(self, N: int, node_type: int):
        self.N, self.n, self.node_type = N, N + 1, node_type
        x, w = nodes_weights(N, node_type)
        D = diff_matrix(x)
        lm, lp = lagrange_at(x, -1.0), lagrange_at(x, 1.0)
        # D_hat_ij = -(w_j / w_i) D_ji ; l_hat = l / w
        Dhat = -(w[None, :] / w[:, None]) * D.T
        self.x_np, self.w_np, self.D_np = x, w, D
        t = lambda a: torch.tensor(a, dtype=DT)
        self.x, self.w, self.D, self.Dhat = t(x), t(w), t(D), t(Dhat)
        self.l_minus, self.l_plus = t(lm), t(lp)
        self.lhat_minus, self.lhat_plus = t(lm / w), t(lp / w)
        # Mortar operators (Sec. "Non-conforming meshes"), a = 0 lower / 1 upper half
        # of a big side, whose nodes sit at eta^a_i = (x_i + 2a - 1)/2 in the big
        # side's coordinate: interpolation I^a_im = l_m(eta^a_i) and the L2
        # projection P^a_i,alpha = l_i(eta^a_alpha) w_alpha / w_i.  Reading: the
        # paper's matrix-vector form swaps the superscripts (U^U = I^L U^B); its
        # element-wise definition, U^L_ij = sum_m U^B_mj l_m(eta^L_i), is used.
        self.I_mortar, self.P_mortar = [], []
        for a in (0, 1):
            V = lagrange_matrix(x, (x + 2 * a - 1) / 2.0)  # V[i, m] = l_m(eta^a_i)
            self.I_mortar.append(t(V))
            self.P_mortar.append(t(V.T * w[None, :] / w[:, None]))

    def l_side(self, sign: int) -> torch.Tensor:
        return self.l_plus if sign > 0 else self.l_minus

    def lhat_side(self, sign: int) -> torch.Tensor:
        return self.lhat_plus if sign > 0 else self.lhat_minus
