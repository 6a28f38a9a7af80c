"""Pins for oracle/qpoint.py: eigen routines, strain, closed-form t = 0 quadrature data."""
import numpy as np
import pytest

from oracle import qpoint
from oracle.hydro import Hydro, Params
from paper_2112_07075_b300 import inputs


def _random_sym(rng, n, d):
    A = rng.standard_normal((n, d, d))
    return 0.5 * (A + np.transpose(A, (0, 2, 1)))


@pytest.mark.parametrize("d", [2, 3])
def test_eig_min_matches_eigh(d):
    rng = np.random.default_rng(1)
    A = _random_sym(rng, 2000, d) * rng.uniform(1e-3, 1e3, size=(2000, 1, 1))
    lam, s = qpoint.eig_min_sym(A)
    w = np.linalg.eigvalsh(A)
    scale = np.abs(w).max(axis=1)
    assert np.max(np.abs(lam - w[:, 0]) / scale) < 5e-14
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0, atol=1e-14)
    res = np.linalg.norm(np.einsum("nij,nj->ni", A, s) - lam[:, None] * s, axis=1)
    assert np.max(res / scale) < 1e-12


def test_eig_min_degenerate_cases():
    A = np.array([np.diag([1.0, 1.0, 2.0]), np.diag([2.0, 1.0, 1.0]), np.zeros((3, 3)),
                  3.0 * np.eye(3), np.diag([-1.0, 4.0, -1.0])])
    lam, s = qpoint.eig_min_sym3(A)
    # The trigonometric closed form loses about half the digits when the two
    # smallest eigenvalues coincide (acos near +1): the error there is O(sqrt(eps)).
    assert np.allclose(lam, [1.0, 1.0, 0.0, 3.0, -1.0], atol=1e-7)
    assert np.allclose(np.linalg.norm(s, axis=1), 1.0)
    for k in range(len(A)):
        assert np.linalg.norm(A[k] @ s[k] - lam[k] * s[k]) < 1e-7
    assert np.array_equal(s[2], [1.0, 0.0, 0.0]) and np.array_equal(s[3], [1.0, 0.0, 0.0])
    lam2, s2 = qpoint.eig_min_sym2(np.array([np.eye(2) * 2.0, np.zeros((2, 2)), np.diag([3.0, -1.0])]))
    assert np.allclose(lam2, [2.0, 0.0, -1.0])
    assert np.array_equal(s2[0], [1.0, 0.0]) and np.array_equal(s2[1], [1.0, 0.0])
    assert abs(abs(s2[2, 1]) - 1.0) < 1e-15


def test_smooth_step():
    e0 = 1e-12
    x = np.array([-1.0, -e0, 0.0, e0, 1.0])
    assert np.allclose(qpoint.smooth_step(x, e0), [0.0, 0.0, 0.5, 1.0, 1.0])


@pytest.mark.parametrize("dim", [2, 3])
def test_affine_velocity_gives_exact_strain(dim):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((dim, dim))
    hy = Hydro(Params(dim=dim, n=2, order=2, q1=3, vertices=inputs.box_vertices(dim, 2, jitter=0.15, seed=2)))
    x = hy.mesh.x0
    v = A @ x
    e = np.ones((hy.mesh.NE, hy.mesh.NL1))
    _, _, ex = hy.qdata(x, v, e)
    assert np.max(np.abs(ex["eps"] - 0.5 * (A + A.T)[None])) < 1e-13
    assert np.max(np.abs(ex["rho"] * ex["detJ"] - hy.rho0detJ0.ravel())) < 1e-15


@pytest.mark.parametrize("dim,n,p", [(2, 4, 2), (3, 2, 3)])
def test_undeformed_mesh_at_rest_closed_form_dt(dim, n, p):
    gamma, cfl, e0 = 5.0 / 3.0, 0.5, 2.0
    hy = Hydro(Params(dim=dim, n=n, order=p, q1=2 * p, vertices=inputs.box_vertices(dim, n),
                      gamma=gamma, cfl=cfl))
    x = hy.mesh.x0
    e = np.full((hy.mesh.NE, hy.mesh.NL1), e0)
    D, dt, ex = hy.qdata(x, np.zeros_like(x), e)
    h = 1.0 / n
    hmin = h / p
    cs = np.sqrt(gamma * (gamma - 1) * e0)
    h0 = h / p                                           # (|Omega|/NE)^(1/d) / p
    mu = 0.5 * 1.0 * h0 * cs                             # lam = 0: linear term on, quadratic 0
    ref = cfl / (cs / hmin + 2.5 * mu / (hmin * hmin))
    assert abs(hy.h0 - h0) < 1e-15
    assert np.allclose(ex["hmin"], hmin, rtol=1e-13)
    assert np.allclose(ex["mu"], mu, rtol=1e-13)
    assert abs(dt - ref) < 1e-13 * ref
    p_ref = (gamma - 1) * e0
    # D = omega detJ sigma J^{-T} = -p omega h^{d-1} I
    w = np.tile(hy.T.w, hy.mesh.NE)
    expect = -p_ref * (w * h ** (dim - 1))[:, None, None] * np.eye(dim)[None]
    assert np.max(np.abs(D.reshape(-1, dim, dim) - expect)) < 1e-14


def test_inverted_element_gives_zero_dt():
    hy = Hydro(Params(dim=2, n=2, order=1, q1=2, vertices=inputs.box_vertices(2, 2)))
    x = hy.mesh.x0.copy()
    x[0, 4] = 1.2                                      # centre node pushed past the right side
    _, dt, ex = hy.qdata(x, np.zeros_like(x), np.ones((4, 1)))
    assert ex["inverted"] and dt == 0.0
