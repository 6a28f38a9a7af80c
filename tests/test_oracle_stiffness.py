"""Pins of the oracle's stiffness operator and discrete Laplacian (Sections 2.1, 3.3, 6).

Each pin is fixed by the continuous problem or a textbook value, not by the
oracle's own formulas: the stiffness of a constant vanishes; the unit-square Q1
element matrix is the classical one; Green's identity makes the interior rows of
S f vanish for linear f (exactly, also on jittered meshes) and equal
-d int w_i dx for f = |x|^2/2; and a field with zero normal derivative whose
Laplacian is in the discrete space has that Laplacian reproduced at every node.
A missing det J, a transposed J^-1, a wrong weight or a sign error fails one of them.
"""
import numpy as np
import pytest

from oracle.fem import Tables
from oracle.mesh import Mesh
from oracle.stiffness import Stiffness
from paper_2112_07075_b300 import inputs


def _interior(mesh):
    """Nodes off every box face (the velocity constraint marks the faces per component)."""
    return np.all(mesh.free, axis=0)


@pytest.mark.parametrize("dim,n,p,q1,jit", [(2, 3, 2, 4, 0.12), (3, 2, 2, 4, 0.12), (2, 2, 4, 8, 0.1)])
def test_stiffness_of_a_constant_vanishes(dim, n, p, q1, jit):
    m = Mesh(inputs.box_vertices(dim, n, jitter=jit, seed=4), dim, n, p)
    st = Stiffness(m, Tables(dim, p, q1), m.x0)
    assert np.max(np.abs(st.S @ np.ones(m.NH1))) <= 1e-13 * abs(st.S).max()


def test_unit_square_q1_element_is_the_textbook_matrix():
    m = Mesh(inputs.box_vertices(2, 1), 2, 1, 1)
    st = Stiffness(m, Tables(2, 1, 2), m.x0)
    # lexicographic nodes (0,0), (1,0), (0,1), (1,1): edge neighbours -1, across -2
    ref = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    assert np.allclose(st.S.toarray(), ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim,n,p,q1", [(2, 4, 1, 2), (2, 3, 2, 4), (2, 3, 3, 6), (3, 3, 1, 2), (3, 3, 2, 4)])
def test_linear_field_has_zero_interior_rows_on_jittered_meshes(dim, n, p, q1):
    m = Mesh(inputs.box_vertices(dim, n, jitter=0.15, seed=6), dim, n, p)
    st = Stiffness(m, Tables(dim, p, q1), m.x0)
    a = np.random.default_rng(1).uniform(-1, 1, dim)
    f = a @ m.x0 + 0.3
    Sf = st.S @ f
    inner = _interior(m)
    assert inner.sum() > 0
    assert np.max(np.abs(Sf[inner])) <= 1e-13 * np.max(np.abs(Sf))
    assert np.max(np.abs(Sf[~inner])) > 1e-3        # boundary flux is there


@pytest.mark.parametrize("dim,n,p,q1", [(2, 3, 2, 4), (2, 2, 4, 8), (3, 2, 2, 4), (3, 2, 3, 6)])
def test_quadratic_field_gives_minus_d_times_the_node_integral(dim, n, p, q1):
    m = Mesh(inputs.box_vertices(dim, n), dim, n, p)
    st = Stiffness(m, Tables(dim, p, q1), m.x0)
    f = 0.5 * np.sum(m.x0 ** 2, axis=0)
    inner = _interior(m)
    node_int = st.M @ np.ones(m.NH1)                  # int w_i dx
    assert np.max(np.abs((st.S @ f)[inner] + dim * node_int[inner])) <= 1e-13


@pytest.mark.parametrize("dim,n,p,q1", [(2, 2, 3, 6), (2, 3, 4, 8), (3, 2, 3, 6)])
def test_laplacian_of_a_neumann_cubic_is_exact(dim, n, p, q1):
    m = Mesh(inputs.box_vertices(dim, n), dim, n, p)
    st = Stiffness(m, Tables(dim, p, q1), m.x0)
    X = m.x0
    f = np.sum(X ** 2 / 2 - X ** 3 / 3, axis=0)
    lap = st.laplacian(np.stack([f, 2.0 * f]))
    exact = np.sum(1.0 - 2.0 * X, axis=0)
    assert np.max(np.abs(lap[0] - exact)) <= 1e-11
    assert np.max(np.abs(lap[1] - 2.0 * exact)) <= 1e-11
