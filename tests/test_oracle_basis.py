"""Pins for oracle/basis.py: quadrature exactness, GLL points, Lagrange bases."""
import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_exact_to_degree_2n_minus_1(n):
    x, w = basis.gauss_legendre(n)
    assert abs(w.sum() - 1.0) < 1e-14
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14, k
    # and not exact one degree higher
    assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-13


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_points_are_lobatto_roots(p):
    z = basis.gll_points(p)
    # interior GLL points on [-1,1] are the roots of P_p'(t), computed here
    # through numpy's Legendre-series routines (an independent route).
    c = np.zeros(p + 1)
    c[p] = 1.0
    interior = np.sort(np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c))) if p > 1 else []
    ref = np.concatenate([[-1.0], interior, [1.0]])
    assert np.allclose(2 * z - 1, ref, atol=1e-15, rtol=0)
    assert np.allclose(z + z[::-1], 1.0, atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gll_weights_closed_form(p):
    # Lobatto weights on [0,1] (textbook closed forms) reproduced by integrating the basis exactly.
    ref = {1: [1 / 2, 1 / 2], 2: [1 / 6, 2 / 3, 1 / 6], 3: [1 / 12, 5 / 12, 5 / 12, 1 / 12],
           4: [1 / 20, 49 / 180, 16 / 45, 49 / 180, 1 / 20]}[p]
    x, w = basis.gauss_legendre(p + 1)
    B = basis.lagrange_values(basis.gll_points(p), x)
    assert np.allclose(w @ B, ref, atol=1e-15, rtol=0)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_delta_unity_and_derivatives(p):
    for nodes in (basis.gll_points(p), basis.gauss_legendre(p)[0]):
        n = nodes.size
        assert np.allclose(basis.lagrange_values(nodes, nodes), np.eye(n), atol=1e-14)
        x = np.linspace(-0.1, 1.1, 17)
        B = basis.lagrange_values(nodes, x)
        G = basis.lagrange_derivs(nodes, x)
        assert np.allclose(B.sum(axis=1), 1.0, atol=1e-13)
        assert np.allclose(G.sum(axis=1), 0.0, atol=1e-11)
        for i in range(n):
            coef = np.polyfit(nodes, np.eye(n)[i], n - 1)
            assert np.allclose(G[:, i], np.polyval(np.polyder(coef), x), atol=1e-10)
            assert np.allclose(B[:, i], np.polyval(coef, x), atol=1e-11)
