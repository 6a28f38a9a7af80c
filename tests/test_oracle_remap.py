"""Pins of the oracle's velocity remap (M(tau) dv/dtau = K(tau) v, Section 3.5).

Each pin comes from what the continuous problem fixes, not from the oracle's own
formulas: the convection of a constant vanishes (K 1 = 0); the mass matrix
integrates 1 to the volume of the box at every pseudo-time; a zero displacement
changes nothing; and a field linear in the physical coordinates is transported
exactly (its discrete advection is exact and the nodal values are linear in tau),
so after the remap its nodal values equal the field at the target nodes. A sign
error in K, a transposed J^-1 or a missing det J breaks the last pin on the
jittered (non-affine) meshes used here.
"""
import numpy as np
import pytest

from oracle.fem import Tables
from oracle.mesh import Mesh
from oracle.remap import Remap
from paper_2112_07075_b300 import inputs


def _meshes(dim, n, p):
    m0 = Mesh(inputs.box_vertices(dim, n, jitter=0.12, seed=1), dim, n, p)
    m1 = Mesh(inputs.box_vertices(dim, n, jitter=0.12, seed=2), dim, n, p)
    return m0, m1


@pytest.mark.parametrize("dim,n,p,q1", [(2, 3, 2, 4), (3, 2, 2, 4), (2, 2, 3, 6)])
def test_convection_of_a_constant_vanishes(dim, n, p, q1):
    m0, m1 = _meshes(dim, n, p)
    R = Remap(m0, Tables(dim, p, q1), m0.x0, m1.x0)
    for tau in (0.0, 0.4, 1.0):
        _, K = R.operators(tau)
        assert np.max(np.abs(K @ np.ones(m0.NH1))) <= 1e-14 * abs(K).max()


@pytest.mark.parametrize("dim,n,p,q1", [(2, 3, 2, 4), (3, 2, 3, 6)])
def test_mass_integrates_one_to_the_box_volume(dim, n, p, q1):
    m0, m1 = _meshes(dim, n, p)
    R = Remap(m0, Tables(dim, p, q1), m0.x0, m1.x0)
    one = np.ones(m0.NH1)
    for tau in (0.0, 0.5, 1.0):
        M, _ = R.operators(tau)
        assert abs(one @ (M @ one) - 1.0) <= 1e-13


def test_zero_displacement_leaves_the_field_unchanged():
    m0, _ = _meshes(2, 3, 2)
    v = inputs.uniform(5, (2, m0.NH1), -1.0, 1.0)
    R = Remap(m0, Tables(2, 2, 4), m0.x0, m0.x0)
    assert np.array_equal(R.remap(v, 2), v)


@pytest.mark.parametrize("dim,n,p,q1,steps", [(2, 3, 1, 2, 1), (2, 3, 2, 4, 2), (3, 2, 2, 4, 2),
                                              (2, 2, 3, 6, 3), (3, 2, 3, 6, 1)])
def test_linear_field_is_remapped_exactly(dim, n, p, q1, steps):
    m0, m1 = _meshes(dim, n, p)
    rng = np.random.default_rng(3)
    A, b = rng.uniform(-1, 1, (dim, dim)), rng.uniform(-1, 1, dim)
    v0 = A @ m0.x0 + b[:, None]
    R = Remap(m0, Tables(dim, p, q1), m0.x0, m1.x0, constrained=False)
    v1 = R.remap(v0, steps)
    exact = A @ m1.x0 + b[:, None]
    assert np.max(np.abs(v1 - exact)) <= 1e-12 * np.max(np.abs(exact))
    # and the field did move: the target differs from the source by far more
    assert np.max(np.abs(exact - v0)) > 1e-3
