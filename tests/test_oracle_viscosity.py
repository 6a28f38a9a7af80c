"""Closed-form pins of the oracle's artificial viscosity (Section 2.1: total stress =
physical stress + a stress due to artificial viscosity) through Hydro.qdata.

The reading pinned here: mu = 2 rho h^2 |lam| + 1/2 rho h c_s (1 - S(lam - 2 eps0)),
lam the smallest eigenvalue of the strain rate eps and s its unit eigenvector,
h = h0 |J J0^{-1} s|, h0 = (|Omega0| / NE)^{1/d} / p, rho = rho0 detJ0 / detJ,
sigma = -p I + mu eps, and the CFL estimate 1/dt = c_s / h_min + 2.5 mu / (rho h_min^2)
with h_min = sigma_min(J) / p.

Every case uses affine meshes and affine velocities, so each quadrature point has
the same J, eps and state, and every expected value below is worked out by hand
from the construction (a chosen rotation R gives the eigenpairs; the mesh maps A0,
A1 give J0, J and the volume). numpy is used only for the matrix products and
norms of those hand values and for a textbook SVD of J.

The planted-error tests load a copy of oracle/qpoint.py with one deliberate
mistake (a coefficient, the order of J and J0^{-1}, the largest instead of the
smallest eigenvalue, a dropped absolute value, the switch of the linear term,
an undeformed length scale) and check that at least one pin fails for each.
"""
import types

import numpy as np
import pytest

import oracle.hydro as hydro_mod
from oracle import qpoint
from oracle.hydro import Hydro, Params
from paper_2112_07075_b300 import inputs

GAMMA, CFL, E_C = 5.0 / 3.0, 0.5, 2.0
TOL = 1e-12


def _rot3(a, b, c):
    ca, sa, cb, sb, cc, sc = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)
    Rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1.0]])
    Ry = np.array([[cb, 0, sb], [0, 1.0, 0], [-sb, 0, cb]])
    Rx = np.array([[1.0, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return Rz @ Ry @ Rx


def _rot2(a):
    return np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])


# Initial-mesh maps (sheared, non-symmetric) and deformations that do not commute with them.
A0 = {2: np.array([[1.0, 0.35], [0.1, 0.8]]),
      3: np.array([[1.0, 0.3, 0.0], [0.0, 0.8, 0.2], [0.1, 0.0, 1.1]])}
A1 = {2: np.array([[1.4, 0.0], [0.25, 0.9]]),
      3: np.array([[1.3, 0.2, 0.0], [0.0, 0.9, 0.1], [0.3, 0.0, 1.0]])}
ROT = {2: _rot2(0.6), 3: _rot3(0.6, -0.4, 0.9)}
# eigenvalues of eps: mixed signs (compression along the first axis of R) and pure expansion
LAM_MIXED = {2: np.array([-2.0, 0.5]), 3: np.array([-2.0, 0.5, -0.7])}
LAM_EXPAND = {2: np.array([0.4, 1.5]), 3: np.array([0.4, 1.0, 1.5])}


def _hydro(dim, n, p, A=None):
    V = inputs.box_vertices(dim, n)
    if A is not None:
        V = V @ A.T
    return Hydro(Params(dim=dim, n=n, order=p, q1=p + 1, vertices=V, gamma=GAMMA, cfl=CFL))


def _expected(dim, n, p, J0, J, lam, s, detA0):
    """Hand evaluation of rho, c_s, h, mu, D per qpoint and dt for one affine case."""
    rho = np.linalg.det(J0) / np.linalg.det(J)              # rho0 = 1
    cs = np.sqrt(GAMMA * (GAMMA - 1.0) * E_C)
    pres = (GAMMA - 1.0) * rho * E_C
    h0 = (detA0 / n ** dim) ** (1.0 / dim) / p               # |Omega0| = det A0 for the unit box
    h = h0 * np.linalg.norm(J @ np.linalg.inv(J0) @ s)
    mu = 2.0 * rho * h * h * abs(lam)
    if lam < 0.0:                                            # compression: linear term on
        mu += 0.5 * rho * h * cs
    hmin = np.linalg.svd(J, compute_uv=False).min() / p
    dt = CFL / (cs / hmin + 2.5 * mu / (rho * hmin * hmin))
    return rho, pres, mu, h, dt


def _run(hy, x, v):
    e = np.full((hy.mesh.NE, hy.mesh.NL1), E_C)
    D, dt, ex = hy.qdata(x, v, e)
    return D, dt, ex


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / max(abs(b), 1e-300))


def case_uniform_compression(dim):
    """v = -alpha x on an undeformed Cartesian mesh: eps = -alpha I, lam = -alpha, J = J0,
    so h = h0 for any eigenvector; mu = 2 h0^2 alpha + h0 c_s / 2 and
    D = -(p + mu alpha) omega h_box^{d-1} I."""
    n, p, alpha = 3, 2, 3.0
    hy = _hydro(dim, n, p)
    x = hy.mesh.x0
    D, dt, ex = _run(hy, x, -alpha * x)
    hb = 1.0 / n
    h0 = hb / p
    cs = np.sqrt(GAMMA * (GAMMA - 1.0) * E_C)
    mu = 2.0 * h0 * h0 * alpha + 0.5 * h0 * cs
    pres = (GAMMA - 1.0) * E_C
    hmin = hb / p
    dt_ref = CFL / (cs / hmin + 2.5 * mu / (hmin * hmin))
    w = np.tile(hy.T.w, hy.mesh.NE)
    D_ref = -(pres + mu * alpha) * (w * hb ** (dim - 1))[:, None, None] * np.eye(dim)[None]
    return max(_rel(ex["mu"], mu), _rel(dt, dt_ref),
               float(np.max(np.abs(D.reshape(-1, dim, dim) - D_ref)) / np.max(np.abs(D_ref))))


def case_stretched_mesh(dim):
    """Cartesian initial mesh stretched by S = diag(2, 1) or diag(2, 5/4, 1) with v_1 = -alpha x_1:
    eps = diag(-alpha, 0, ..), s = e_1, h = h0 |S e_1| = 2 h0, rho = 1 / det S. (The 3D stretch
    keeps the singular values of J distinct: the trigonometric eigenvalue form loses about
    half the digits of sigma_min at a double smallest eigenvalue of J^T J.)"""
    n, p, alpha = 2, 2, 1.5
    hy = _hydro(dim, n, p)
    S = np.diag([2.0, 1.0] if dim == 2 else [2.0, 1.25, 1.0])
    x = S @ hy.mesh.x0
    v = np.zeros_like(x)
    v[0] = -alpha * x[0]
    D, dt, ex = _run(hy, x, v)
    h0 = (1.0 / n) / p
    h, rho = 2.0 * h0, 1.0 / (2.0 if dim == 2 else 2.5)
    cs = np.sqrt(GAMMA * (GAMMA - 1.0) * E_C)
    mu = 2.0 * rho * h * h * alpha + 0.5 * rho * h * cs
    hmin = (1.0 / n) / p                                      # sigma_min(S h_box) = h_box
    dt_ref = CFL / (cs / hmin + 2.5 * mu / (rho * hmin * hmin))
    return max(_rel(ex["mu"], mu), _rel(dt, dt_ref))


def case_affine(dim, lams):
    """Sheared initial mesh x0 = A0 X, current positions x = A1 x0, velocity v = eps x with
    eps = R diag(lams) R^T: J0 = A0 h_box, J = A1 A0 h_box, s = the column of R of the
    smallest eigenvalue, h = h0 |A1 s|."""
    n, p = 2, 2
    A0m, A1m, R = A0[dim], A1[dim], ROT[dim]
    hy = _hydro(dim, n, p, A0m)
    x = A1m @ hy.mesh.x0
    eps = R @ np.diag(lams) @ R.T
    D, dt, ex = _run(hy, x, eps @ x)
    hb = 1.0 / n
    k = int(np.argmin(lams))
    J0, J = A0m * hb, A1m @ A0m * hb
    rho, pres, mu, h, dt_ref = _expected(dim, n, p, J0, J, lams[k], R[:, k], np.linalg.det(A0m))
    sigma = -pres * np.eye(dim) + mu * eps
    w = np.tile(hy.T.w, hy.mesh.NE)
    D_ref = (w * np.linalg.det(J))[:, None, None] * (sigma @ np.linalg.inv(J).T)[None]
    return max(_rel(ex["mu"], mu), _rel(ex["rho"], rho), _rel(dt, dt_ref),
               float(np.max(np.abs(D.reshape(-1, dim, dim) - D_ref)) / np.max(np.abs(D_ref))))


def _all_cases(dim):
    return {"uniform_compression": case_uniform_compression(dim),
            "stretched_mesh": case_stretched_mesh(dim),
            "affine_mixed": case_affine(dim, LAM_MIXED[dim]),
            "affine_expansion": case_affine(dim, LAM_EXPAND[dim])}


@pytest.mark.parametrize("dim", [2, 3])
def test_viscosity_closed_forms(dim):
    errs = _all_cases(dim)
    assert all(e < TOL for e in errs.values()), errs


@pytest.mark.parametrize("dim", [2, 3])
def test_pins_are_sensitive(dim):
    """The construction makes the wrong readings give different numbers: J J0^{-1} and
    J0^{-1} J differ on s, and the largest eigenvalue differs from the smallest."""
    A0m, A1m, R = A0[dim], A1[dim], ROT[dim]
    s = R[:, 0]
    a = np.linalg.norm(A1m @ s)
    b = np.linalg.norm(np.linalg.inv(A0m) @ A1m @ A0m @ s)
    assert abs(a - b) > 1e-2 * a
    assert LAM_MIXED[dim].min() < 0.0 < LAM_MIXED[dim].max()


# (description, original text in oracle/qpoint.py, planted replacement)
PLANTS = [
    ("quadratic coefficient 1 instead of 2", "mu = 2.0 * rho * h * h * np.abs(lam)",
     "mu = 1.0 * rho * h * h * np.abs(lam)"),
    ("J0^{-1} J instead of J J0^{-1}", 'hvec = np.einsum("ncl,nlb,nb->nc", J, Jinv0, s)',
     'hvec = np.einsum("ncl,nlb,nb->nc", Jinv0, J, s)'),
    ("largest eigenvalue (3D)", "np.cos(phi + 2.0 * np.pi / 3.0)", "np.cos(phi)"),
    ("largest eigenvalue (2D)", "lam = 0.5 * (a + c) - np.sqrt", "lam = 0.5 * (a + c) + np.sqrt"),
    ("no absolute value", "h * h * np.abs(lam)", "h * h * lam"),
    ("linear term switched by -lam", "smooth_step(lam - 2.0 * EPS0, EPS0)", "smooth_step(-lam - 2.0 * EPS0, EPS0)"),
    ("undeformed length scale", "h = h0 * np.linalg.norm(hvec, axis=1)", "h = h0 * np.linalg.norm(s, axis=1)"),
    ("linear coefficient 1 instead of 1/2", "+ 0.5 * rho * h * cs", "+ 1.0 * rho * h * cs"),
]


def _planted_qdata(old, new):
    src = open(qpoint.__file__).read()
    assert src.count(old) == 1, f"pin target not found in oracle/qpoint.py: {old}"
    mod = types.ModuleType("qpoint_planted")
    exec(compile(src.replace(old, new), "qpoint_planted", "exec"), mod.__dict__)
    return mod.qdata


@pytest.mark.parametrize("desc,old,new", PLANTS, ids=[p[0] for p in PLANTS])
def test_planted_error_fails_a_pin(monkeypatch, desc, old, new):
    monkeypatch.setattr(hydro_mod, "qpoint_qdata", _planted_qdata(old, new))
    dims = [2] if "2D" in desc else [3] if "3D" in desc else [2, 3]
    for dim in dims:
        errs = _all_cases(dim)
        assert max(errs.values()) > 1e-6, (desc, dim, errs)
