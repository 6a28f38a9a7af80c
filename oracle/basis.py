"""1D node sets, quadrature rules and Lagrange bases on the reference interval [0, 1].

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings (the paper names tensor-product bases on quads/hexes, Section 3.2, but
fixes neither nodes nor quadrature):
  * H1 (continuous) space Q_p: Lagrange basis on the p+1 Gauss-Lobatto-Legendre
    (GLL) points; closed forms for p <= 4.
  * L2 (discontinuous) space Q_{p-1}: Lagrange basis on the p Gauss-Legendre points.
  * Quadrature: the Q1-point Gauss-Legendre rule per direction.

Pins (tests/test_oracle_basis.py): GL exactness on monomials up to degree
2*Q1-1 and failure at 2*Q1; GLL points are the roots of (1-t^2) P_p'(t) (via a
separate Legendre-series route); nodal delta property; partition of unity;
derivative rows sum to zero; derivatives agree with exact polynomial
differentiation of the interpolant (numpy.polynomial fit through the nodes).
"""
from __future__ import annotations

import math

import numpy as np


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule mapped to [0, 1]: (points, weights)."""
    if n < 1:
        raise ValueError("need n >= 1")
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def gll_points(p: int) -> np.ndarray:
    """The p+1 Gauss-Lobatto-Legendre points on [0, 1] (closed forms for p <= 4)."""
    if p == 1:
        return np.array([0.0, 1.0])
    if p == 2:
        return np.array([0.0, 0.5, 1.0])
    if p == 3:
        a = 1.0 / math.sqrt(5.0)
        return np.array([0.0, 0.5 * (1.0 - a), 0.5 * (1.0 + a), 1.0])
    if p == 4:
        a = math.sqrt(3.0 / 7.0)
        return np.array([0.0, 0.5 * (1.0 - a), 0.5, 0.5 * (1.0 + a), 1.0])
    raise ValueError("GLL points implemented for 1 <= p <= 4")


def lagrange_values(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """B[k, i] = l_i(x_k), the i-th Lagrange polynomial on `nodes` evaluated at x_k."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = nodes.size
    B = np.ones((x.size, n))
    for i in range(n):
        for m in range(n):
            if m != i:
                B[:, i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
    return B


def lagrange_derivs(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """G[k, i] = l_i'(x_k) by the product rule: sum over the factor that is differentiated."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    n = nodes.size
    G = np.zeros((x.size, n))
    for i in range(n):
        for m in range(n):
            if m == i:
                continue
            term = np.full(x.size, 1.0 / (nodes[i] - nodes[m]))
            for k in range(n):
                if k != i and k != m:
                    term *= (x - nodes[k]) / (nodes[i] - nodes[k])
            G[:, i] += term
    return G


class Basis1D:
    """All 1D tables for one (order p, quadrature points per direction Q1) pair.

    B[q, i] = w_i(xi_q), G[q, i] = w_i'(xi_q) for the H1 basis (p+1 functions);
    Bl[q, j] = phi_j(xi_q) for the L2 basis (p functions); xq, wq = GL rule.
    """

    def __init__(self, p: int, q1: int):
        if p < 1 or p > 4:
            raise ValueError("order must be in 1..4")
        self.p = p
        self.q1 = q1
        self.d1 = p + 1
        self.l1 = p
        self.xq, self.wq = gauss_legendre(q1)
        self.h1_nodes = gll_points(p)
        self.l2_nodes, _ = gauss_legendre(p)
        self.B = lagrange_values(self.h1_nodes, self.xq)
        self.G = lagrange_derivs(self.h1_nodes, self.xq)
        self.Bl = lagrange_values(self.l2_nodes, self.xq)
