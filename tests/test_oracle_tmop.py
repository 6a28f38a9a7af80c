"""Pins of the oracle's TMOP objective and derivatives (Section 2.2, Section 3.4 Eqs. 6-7).

The metric is pinned by closed-form values, each derivative level by central
differences of the level below (metric -> first -> second derivative; objective ->
gradient -> Hessian action) on jittered meshes, and the assembled Hessian by its
symmetry. An ideal mesh (uniform, W = h I) is a minimiser of the metric term:
the term and its gradient vanish there. A wrong sign, index, transposed W^-1 or a
dropped term in any formula fails one of these.
"""
import numpy as np
import pytest

from oracle.fem import Tables
from oracle.mesh import Mesh
from oracle.tmop import Tmop, d2mu, dmu, mu
from paper_2112_07075_b300 import inputs


def _rot(dim, ang):
    if dim == 2:
        c, s = np.cos(ang), np.sin(ang)
        return np.array([[c, -s], [s, c]])
    a, b = ang, 0.7 * ang
    Rz = np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, np.cos(b), -np.sin(b)], [0, np.sin(b), np.cos(b)]])
    return Rz @ Rx


@pytest.mark.parametrize("dim", [2, 3])
def test_metric_closed_forms(dim):
    assert abs(mu(np.eye(dim))) < 1e-15
    assert abs(mu(2.5 * _rot(dim, 0.4))) < 1e-14           # scaled rotation: ideal shape
    S = np.diag([2.0] + [1.0] * (dim - 1))                   # stretched by 2 along x
    expect = 5.0 / 4.0 - 1.0 if dim == 2 else 6.0 / (3.0 * 2.0 ** (2.0 / 3.0)) - 1.0
    assert abs(mu(S) - expect) < 1e-15
    assert mu(S) > 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_metric_derivatives_match_central_differences(dim):
    rng = np.random.default_rng(dim)
    T = np.eye(dim) + 0.3 * rng.uniform(-1, 1, (dim, dim))
    assert np.linalg.det(T) > 0
    h = 1e-6
    fd1 = np.zeros((dim, dim))
    fd2 = np.zeros((dim, dim, dim, dim))
    for b in range(dim):
        for p in range(dim):
            E = np.zeros((dim, dim))
            E[b, p] = h
            fd1[b, p] = (mu(T + E) - mu(T - E)) / (2 * h)
            fd2[:, :, b, p] = (dmu(T + E) - dmu(T - E)) / (2 * h)
    assert np.max(np.abs(dmu(T) - fd1)) < 1e-8
    assert np.max(np.abs(d2mu(T) - fd2)) < 1e-7
    H = d2mu(T).reshape(dim * dim, dim * dim)
    assert np.max(np.abs(H - H.T)) < 1e-13


def _tmop(dim, n, p, q1, jit=0.15, seed=7):
    m = Mesh(inputs.box_vertices(dim, n, jitter=jit, seed=seed), dim, n, p)
    T = Tables(dim, p, q1)
    h = 1.0 / n
    x0 = Mesh(inputs.box_vertices(dim, n), dim, n, p).x0
    # a general (non-symmetric) target matrix, so that every use of W^-1 is pinned
    W = h * (np.eye(dim) + np.array([[0.0, 0.2, 0.1], [-0.1, 0.05, 0.0], [0.15, 0.0, -0.1]])[:dim, :dim])
    return m, Tmop(m, T, W, x0, gamma=0.3, dlim=0.5 * h)


@pytest.mark.parametrize("dim,n,p,q1", [(2, 3, 1, 2), (2, 2, 2, 4), (2, 2, 3, 6), (3, 2, 1, 2), (3, 2, 2, 4)])
def test_gradient_matches_central_differences_of_the_objective(dim, n, p, q1):
    m, tm = _tmop(dim, n, p, q1)
    x = m.x0
    g = tm.gradient(x)
    rng = np.random.default_rng(11)
    h = 1e-6
    for _ in range(6):
        a, i = rng.integers(0, dim), rng.integers(0, m.NH1)
        xp, xm = x.copy(), x.copy()
        xp[a, i] += h
        xm[a, i] -= h
        fd = (tm.objective(xp) - tm.objective(xm)) / (2 * h)
        assert abs(fd - g[a, i]) <= 1e-6 * max(1.0, np.max(np.abs(g)))
    # and in a random direction (covers every entry at once)
    u = rng.uniform(-1, 1, x.shape)
    fd = (tm.objective(x + h * u) - tm.objective(x - h * u)) / (2 * h)
    assert abs(fd - np.sum(g * u)) <= 1e-6 * np.sum(np.abs(g * u))


@pytest.mark.parametrize("dim,n,p,q1", [(2, 3, 1, 2), (2, 2, 2, 4), (2, 2, 3, 6), (3, 2, 1, 2), (3, 2, 2, 4)])
def test_hessian_matches_central_differences_of_the_gradient(dim, n, p, q1):
    m, tm = _tmop(dim, n, p, q1)
    x = m.x0
    rng = np.random.default_rng(12)
    u = rng.uniform(-1, 1, x.shape)
    h = 1e-6
    fd = (tm.gradient(x + h * u) - tm.gradient(x - h * u)) / (2 * h)
    Hu = tm.hessian_mult(x, u)
    assert np.max(np.abs(Hu - fd)) <= 1e-6 * np.max(np.abs(Hu))
    H = tm.hessian(x)
    assert abs(H - H.T).max() <= 1e-12 * abs(H).max()
    assert np.array_equal(tm.hessian_diag(x).ravel(), H.diagonal())


@pytest.mark.parametrize("dim,n,p,q1", [(2, 3, 2, 4), (3, 2, 2, 4), (3, 2, 3, 6)])
def test_ideal_mesh_minimises_the_metric_term(dim, n, p, q1):
    m = Mesh(inputs.box_vertices(dim, n), dim, n, p)
    tm = Tmop(m, Tables(dim, p, q1), np.eye(dim) / n, m.x0, gamma=0.0, dlim=1.0)
    assert abs(tm.objective(m.x0)) < 1e-13
    assert np.max(np.abs(tm.gradient(m.x0))) < 1e-13
    # the Hessian there is positive semi-definite (a minimum): u^T H u >= 0
    rng = np.random.default_rng(5)
    H = tm.hessian(m.x0)
    for _ in range(5):
        u = rng.uniform(-1, 1, dim * m.NH1)
        assert u @ (H @ u) >= -1e-12
