"""Pins for oracle/mesh.py: node positions, restriction table, boundary masks."""
import itertools

import numpy as np
import pytest

from oracle import basis
from oracle.mesh import Mesh
from paper_2112_07075_b300 import inputs


@pytest.mark.parametrize("dim,n,p", [(2, 3, 2), (2, 2, 4), (3, 2, 2), (3, 2, 3)])
def test_nodes_on_uniform_box_are_the_gll_grid(dim, n, p):
    lo, hi = -0.5, 0.5
    m = Mesh(inputs.box_vertices(dim, n, lo, hi), dim, n, p)
    z = basis.gll_points(p)
    h = (hi - lo) / n
    g1 = np.array([lo + h * (e + z[i]) for e in range(n) for i in range(p)] + [hi])
    grid = np.array(list(itertools.product(range(m.N1), repeat=dim)))[:, ::-1]
    gidx = sum(grid[:, a] * m.N1 ** a for a in range(dim))
    for a in range(dim):
        assert np.allclose(m.x0[a, gidx], g1[grid[:, a]], atol=1e-15)


@pytest.mark.parametrize("dim,n,p", [(2, 2, 2), (2, 3, 1), (3, 2, 2)])
def test_restriction_matches_brute_force_lookup(dim, n, p):
    V = inputs.box_vertices(dim, n, jitter=0.2, seed=5)
    m = Mesh(V, dim, n, p)
    z = basis.gll_points(p)
    # brute force: evaluate each element's multilinear map at its local GLL nodes
    # and find the unique global node at that position.
    for e in range(m.NE):
        ec = [(e // n ** a) % n for a in range(dim)]
        for i in range(m.ND1):
            ic = [(i // (p + 1) ** a) % (p + 1) for a in range(dim)]
            pos = np.zeros(dim)
            for corner in itertools.product((0, 1), repeat=dim):
                w = 1.0
                vi = 0
                for a in range(dim):
                    w *= z[ic[a]] if corner[a] else 1.0 - z[ic[a]]
                    vi += (ec[a] + corner[a]) * (n + 1) ** a
                pos += w * V[vi]
            dist = np.linalg.norm(m.x0.T - pos[None, :], axis=1)
            assert np.argmin(dist) == m.e2n[e, i]
            assert dist.min() < 1e-14


@pytest.mark.parametrize("dim,n,p", [(2, 4, 2), (3, 3, 3)])
def test_boundary_mask_counts(dim, n, p):
    m = Mesh(inputs.box_vertices(dim, n), dim, n, p)
    for c in range(dim):
        assert np.sum(~m.free[c]) == 2 * m.N1 ** (dim - 1)
        # constrained nodes of component c lie on the faces normal to axis c
        pos = m.x0[c, ~m.free[c]]
        assert np.all((np.abs(pos) < 1e-15) | (np.abs(pos - 1) < 1e-15))


def test_jitter_keeps_box_faces():
    V = inputs.box_vertices(3, 4, jitter=0.15, seed=3)
    U = inputs.box_vertices(3, 4)
    on_bnd = np.any((U == 0.0) | (U == 1.0), axis=1)
    assert np.array_equal(V[on_bnd], U[on_bnd])
    assert np.max(np.abs(V - U)) <= 0.15 / 4 + 1e-15
    assert np.max(np.abs(V - U)) > 0.1 / 4
