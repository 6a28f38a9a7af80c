"""Pins for oracle/fem.py: mass and force assembly against closed forms and brute force."""
import itertools

import numpy as np
import pytest
import sympy

from oracle import basis
from oracle.fem import Tables, assemble_force, assemble_mass, energy_mass, force_element, jacobians
from oracle.hydro import Hydro, Params
from oracle.mesh import Mesh
from paper_2112_07075_b300 import inputs


def _sympy_gll(p):
    s5, s37 = sympy.sqrt(5), sympy.sqrt(sympy.Rational(3, 7))
    half = sympy.Rational(1, 2)
    return {1: [0, 1], 2: [0, half, 1], 3: [0, half * (1 - 1 / s5), half * (1 + 1 / s5), 1],
            4: [0, half * (1 - s37), half, half * (1 + s37), 1]}[p]


def _exact_1d_mass(p):
    t = sympy.Symbol("t")
    z = _sympy_gll(p)
    L = []
    for i in range(p + 1):
        f = sympy.Integer(1)
        for m in range(p + 1):
            if m != i:
                f *= (t - z[m]) / (z[i] - z[m])
        L.append(sympy.expand(f))
    M = np.array([[float(sympy.integrate(L[i] * L[j], (t, 0, 1))) for j in range(p + 1)]
                  for i in range(p + 1)])
    return M


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 2), (3, 3)])
def test_affine_element_mass_is_kronecker_of_exact_1d(dim, p):
    h = 0.37
    m = Mesh(inputs.box_vertices(dim, 1, 0.0, h), dim, 1, p)
    T = Tables(dim, p, p + 1)                       # exact for degree 2p
    J = jacobians(T, m.gather(m.x0))
    M = assemble_mass(m, T, np.linalg.det(J)).toarray()
    M1 = _exact_1d_mass(p)
    ref = M1
    for _ in range(dim - 1):
        ref = np.kron(M1, ref)
    # global numbering of a single element equals its local numbering
    assert np.allclose(M, h ** dim * ref, rtol=0, atol=1e-15)


def test_total_mass_equals_volume_on_jittered_mesh():
    for dim, p in [(2, 3), (3, 2)]:
        m = Mesh(inputs.box_vertices(dim, 3, jitter=0.2, seed=7), dim, 3, p)
        T = Tables(dim, p, 2 * p)
        detJ = np.linalg.det(jacobians(T, m.gather(m.x0)))
        M = assemble_mass(m, T, 2.5 * detJ)
        assert abs(M.sum() - 2.5) < 1e-13
        Me = energy_mass(T, 2.5 * detJ)
        assert abs(Me.sum() - 2.5) < 1e-13


def test_brute_force_element_mass_one_jittered_element():
    dim, p, q1 = 3, 2, 3
    V = inputs.box_vertices(dim, 1, jitter=0.0)
    V[7] += np.array([0.1, -0.05, 0.2])             # move one corner: non-affine element
    m = Mesh(V, dim, 1, p)
    T = Tables(dim, p, q1)
    detJ = np.linalg.det(jacobians(T, m.gather(m.x0)))[0]
    M = assemble_mass(m, T, detJ[None, :]).toarray()
    b = basis.Basis1D(p, q1)
    D1 = p + 1
    for i in range(D1 ** 3):
        for j in range(D1 ** 3):
            ii = (i % D1, (i // D1) % D1, i // D1 ** 2)
            jj = (j % D1, (j // D1) % D1, j // D1 ** 2)
            s = 0.0
            for qz, qy, qx in itertools.product(range(q1), repeat=3):
                q = qx + q1 * (qy + q1 * qz)
                wi = b.B[qx, ii[0]] * b.B[qy, ii[1]] * b.B[qz, ii[2]]
                wj = b.B[qx, jj[0]] * b.B[qy, jj[1]] * b.B[qz, jj[2]]
                s += b.wq[qx] * b.wq[qy] * b.wq[qz] * detJ[q] * wi * wj
            assert abs(M[i, j] - s) < 1e-15


def test_force_columns_sum_to_zero_momentum():
    for dim, p in [(2, 2), (3, 2), (2, 4)]:
        m = Mesh(inputs.box_vertices(dim, 2, jitter=0.1, seed=1), dim, 2, p)
        T = Tables(dim, p, 2 * p)
        rng = np.random.default_rng(0)
        D = rng.standard_normal((m.NE, T.nq, dim, dim))
        F = assemble_force(m, T, D).toarray().reshape(dim, m.NH1, m.NL2)
        assert np.max(np.abs(F.sum(axis=1))) < 1e-12 * np.max(np.abs(F))


GLL_W = {1: [1 / 2, 1 / 2], 2: [1 / 6, 2 / 3, 1 / 6], 3: [1 / 12, 5 / 12, 5 / 12, 1 / 12],
         4: [1 / 20, 49 / 180, 16 / 45, 49 / 180, 1 / 20]}


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3), (3, 2), (3, 4)])
def test_uniform_pressure_force_is_boundary_traction(dim, p):
    """-F.1 = p * (surface integral of w_i n_c): closed form with textbook GLL weights."""
    L, pres, gamma = 0.8, 2.5, 5.0 / 3.0
    prm = Params(dim=dim, n=1, order=p, q1=p + 2, vertices=inputs.box_vertices(dim, 1, 0.0, L),
                 gamma=gamma, use_viscosity=True)
    hy = Hydro(prm)
    x = hy.mesh.x0
    v = np.zeros_like(x)
    e = np.full((1, p ** dim), pres / (gamma - 1.0))
    D, _, _ = hy.qdata(x, v, e)
    f = -(hy.force_matrix(D) @ np.ones(hy.mesh.NL2)).reshape(dim, -1)
    D1 = p + 1
    for c in range(dim):
        for i in range(D1 ** dim):
            ic = [(i // D1 ** a) % D1 for a in range(dim)]
            sign = (ic[c] == p) - (ic[c] == 0)
            area = np.prod([L * GLL_W[p][ic[a]] for a in range(dim) if a != c])
            assert abs(f[c, i] - pres * sign * area) < 1e-13


@pytest.mark.parametrize("dim,p", [(2, 2), (3, 3)])
def test_force_transpose_on_v_equal_x(dim, p):
    """grad v = I (v = x) without viscosity: (F^T v)_j = -d p int phi_j (GL weights)."""
    L, pres, gamma = 1.3, 0.7, 1.4
    prm = Params(dim=dim, n=1, order=p, q1=p + 1, vertices=inputs.box_vertices(dim, 1, 0.0, L),
                 gamma=gamma, use_viscosity=False)
    hy = Hydro(prm)
    x = hy.mesh.x0
    e = np.full((1, p ** dim), pres / (gamma - 1.0))
    D, _, _ = hy.qdata(x, x, e)
    g = hy.force_matrix(D).T @ x.ravel()
    _, wgl = basis.gauss_legendre(p)
    for j in range(p ** dim):
        jc = [(j // p ** a) % p for a in range(dim)]
        ref = -dim * pres * np.prod([L * wgl[jc[a]] for a in range(dim)])
        assert abs(g[j] - ref) < 1e-13


def test_force_element_equals_quadrature_of_definition():
    """One element, one qpoint term at a time: F_e is linear in D with the stated kernel."""
    dim, p, q1 = 2, 2, 3
    T = Tables(dim, p, q1)
    D = np.zeros((1, T.nq, dim, dim))
    q, c, l = 4, 1, 0
    D[0, q, c, l] = 1.0
    Fe = force_element(T, D)[0]
    expect = np.zeros_like(Fe)
    expect[c] = np.outer(T.G[l, q], T.Bl[q])
    assert np.array_equal(Fe, expect)
