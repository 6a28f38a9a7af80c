"""Quadrature-point physics: geometry, density, ideal-gas EOS, artificial viscosity,
stress, force quadrature data and the time-step estimate.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper (Section 2.1) says only that the total stress is the physical stress
plus a stress due to artificial viscosity, and (Section 6) that quadrature-point
data, artificial-viscosity coefficients and the time step are computed per
quadrature point; it refers the formulas to its citations. The readings below
(single material, ideal gas, tensor viscosity) are:

  density     rho = rho0 detJ0 / detJ                         (Eq. 16, rho|J| = rho0|J0|)
  EOS         e+ = max(e, 0), p = (gamma-1) rho e+, cs = sqrt(gamma (gamma-1) e+)
  strain      eps = sym(grad v), grad v = dV J^{-1}
  viscosity   lam, s = smallest eigenvalue of eps and its unit eigenvector
              h  = h0 |J J0^{-1} s|
              mu = 2 rho h^2 |lam| + 0.5 rho h cs (1 - S(lam - 2 eps0; eps0)),
              S(x; e0) = y^2 (3 - 2y), y = clamp((x + e0) / (2 e0), 0, 1), eps0 = 1e-12
  stress      sigma = -p I + mu eps
  force data  D[c,l] = omega detJ sum_b sigma[c,b] Jinv[l,b]
  time step   hmin = sigma_min(J) / p_order,
              1/dt_q = cs / hmin + 2.5 mu / (rho hmin^2),
              dt_est = CFL / max_q (1/dt_q); dt_est = 0 if any detJ <= 0

Eigen routines (reading of the silent parts): 2D closed form; 3D the
trigonometric closed form for symmetric 3x3 matrices (O. K. Smith, "Eigenvalues
of a symmetric 3x3 matrix", CACM 4(4), 1961). Eigenvector of the smallest
eigenvalue: the largest-norm cross product of two rows of (A - lam I) (3D) or
the largest-norm row rotated by 90 degrees (2D); tie-breaks as in the docstrings.
The trigonometric form is accurate to O(eps * p^2 / gap) in the smallest
eigenvalue, where gap is its distance to the middle one: at an exact double
smallest eigenvalue about half the digits are lost (acos near +1).

Pins (tests/test_oracle_qpoint.py): eigenvalues and eigenvector residuals vs
numpy.linalg.eigh on random and degenerate matrices; an affine velocity v = A x
gives eps = sym(A) exactly; an undeformed Cartesian mesh at t = 0 gives J = h I,
hmin = h / p and the closed-form dt; rho detJ = rho0 detJ0.
Viscosity pins (tests/test_oracle_viscosity.py), each value worked out by hand
from an affine construction: uniform compression v = -alpha x (mu = 2 h0^2 alpha
+ h0 c_s / 2, D, dt); a stretched mesh with v_1 = -alpha x_1 (h = 2 h0, rho < 1);
a sheared initial mesh moved by a non-commuting affine map with a strain rate of
chosen eigenpairs of mixed sign (h = h0 |J J0^{-1} s|, mu, rho, D, dt) and of pure
expansion (linear term off). Each of eight planted mistakes (coefficients 1 for
2 and for 1/2, J0^{-1} J, the largest eigenvalue in 2D and 3D, a dropped absolute
value, the linear-term switch on -lam, an undeformed length scale) fails a pin.
Still fixed by the reading only (parity unpinned by the paper): the choice of
eigenvector inside an eigenspace of dimension > 1 and the constants 1e-12 / 2.5
themselves (the pins fix the formula as read, not that the paper means it).
"""
from __future__ import annotations

import numpy as np

EPS0 = 1.0e-12
DEGEN = 1.0e-14


def smooth_step(x: np.ndarray, e0: float) -> np.ndarray:
    y = np.clip((x + e0) / (2.0 * e0), 0.0, 1.0)
    return y * y * (3.0 - 2.0 * y)


def eig_min_sym2(A: np.ndarray, want_vec: bool = True):
    """Smallest eigenvalue (and unit eigenvector) of symmetric 2x2 matrices A[N,2,2]."""
    a, b, c = A[:, 0, 0], 0.5 * (A[:, 0, 1] + A[:, 1, 0]), A[:, 1, 1]
    lam = 0.5 * (a + c) - np.sqrt(0.25 * (a - c) ** 2 + b * b)
    if not want_vec:
        return lam, None
    r0 = np.stack([a - lam, b], axis=1)
    r1 = np.stack([b, c - lam], axis=1)
    n0 = np.linalg.norm(r0, axis=1)
    n1 = np.linalg.norm(r1, axis=1)
    r = np.where((n0 >= n1)[:, None], r0, r1)
    nr = np.maximum(n0, n1)
    normA = np.sqrt(a * a + 2 * b * b + c * c)
    degen = nr <= DEGEN * normA
    s = np.stack([-r[:, 1], r[:, 0]], axis=1) / np.where(degen, 1.0, nr)[:, None]
    s[degen] = np.array([1.0, 0.0])
    return lam, s


def eig_min_sym3(A: np.ndarray, want_vec: bool = True):
    """Smallest eigenvalue (and unit eigenvector) of symmetric 3x3 matrices A[N,3,3]."""
    A = 0.5 * (A + np.transpose(A, (0, 2, 1)))
    q = (A[:, 0, 0] + A[:, 1, 1] + A[:, 2, 2]) / 3.0
    p1 = A[:, 0, 1] ** 2 + A[:, 0, 2] ** 2 + A[:, 1, 2] ** 2
    p2 = (A[:, 0, 0] - q) ** 2 + (A[:, 1, 1] - q) ** 2 + (A[:, 2, 2] - q) ** 2 + 2.0 * p1
    pp = np.sqrt(p2 / 6.0)
    I = np.eye(3)[None]
    safe = np.where(pp > 0.0, pp, 1.0)
    Bm = (A - q[:, None, None] * I) / safe[:, None, None]
    r = np.clip(0.5 * np.linalg.det(Bm), -1.0, 1.0)
    phi = np.arccos(r) / 3.0
    lam = np.where(pp > 0.0, q + 2.0 * pp * np.cos(phi + 2.0 * np.pi / 3.0), q)
    if not want_vec:
        return lam, None
    M = A - lam[:, None, None] * I
    rows = [M[:, 0, :], M[:, 1, :], M[:, 2, :]]
    cands = [np.cross(rows[0], rows[1]), np.cross(rows[0], rows[2]), np.cross(rows[1], rows[2])]
    norms = np.stack([np.linalg.norm(c, axis=1) for c in cands], axis=1)
    k = np.argmax(norms, axis=1)                       # first maximum on ties
    cbest = np.stack(cands, axis=1)[np.arange(A.shape[0]), k]
    nbest = norms[np.arange(A.shape[0]), k]
    normM2 = np.sum(M * M, axis=(1, 2))
    normA = np.sqrt(np.sum(A * A, axis=(1, 2)))
    s = cbest / np.where(nbest > 0, nbest, 1.0)[:, None]
    degen = nbest <= DEGEN * normM2
    if np.any(degen):
        for n in np.nonzero(degen)[0]:
            normMn = np.sqrt(normM2[n])
            if normMn <= DEGEN * normA[n] or normMn == 0.0:
                s[n] = np.array([1.0, 0.0, 0.0])        # A = lam I: any direction
            else:
                rn = np.array([np.linalg.norm(rows[i][n]) for i in range(3)])
                rv = rows[int(np.argmax(rn))][n]
                kk = int(np.argmin(np.abs(rv)))
                ek = np.zeros(3)
                ek[kk] = 1.0
                c = np.cross(rv, ek)
                s[n] = c / np.linalg.norm(c)
    return lam, s


def eig_min_sym(A: np.ndarray, want_vec: bool = True):
    return eig_min_sym2(A, want_vec) if A.shape[-1] == 2 else eig_min_sym3(A, want_vec)


def qdata(J, Jinv0, dV, e_q, rho0detJ0, w, *, gamma, cfl, order, h0, use_viscosity):
    """Per-qpoint physics. Arrays are [N, ...] over all quadrature points.

    J, Jinv0, dV: [N, d, d]; e_q, rho0detJ0 (without the weight), w: [N].
    Returns (D [N,d,d], dt_est, dict of intermediates).
    """
    N, d, _ = J.shape
    detJ = np.linalg.det(J)
    inverted = bool(np.any(detJ <= 0.0))
    Jinv = np.linalg.inv(np.where((detJ > 0)[:, None, None], J, np.eye(d)[None]))
    rho = rho0detJ0 / np.where(detJ > 0, detJ, 1.0)
    ep = np.maximum(e_q, 0.0)
    pres = (gamma - 1.0) * rho * ep
    cs = np.sqrt(gamma * (gamma - 1.0) * ep)
    grad = np.einsum("ncl,nlb->ncb", dV, Jinv)
    eps = 0.5 * (grad + np.transpose(grad, (0, 2, 1)))
    sigma = -pres[:, None, None] * np.eye(d)[None]
    mu = np.zeros(N)
    if use_viscosity:
        lam, s = eig_min_sym(eps, True)
        hvec = np.einsum("ncl,nlb,nb->nc", J, Jinv0, s)
        h = h0 * np.linalg.norm(hvec, axis=1)
        mu = 2.0 * rho * h * h * np.abs(lam) + 0.5 * rho * h * cs * (1.0 - smooth_step(lam - 2.0 * EPS0, EPS0))
        sigma = sigma + mu[:, None, None] * eps
    D = (w * detJ)[:, None, None] * np.einsum("ncb,nlb->ncl", sigma, Jinv)
    JtJ = np.einsum("nlc,nlb->ncb", J, J)
    lamJ, _ = eig_min_sym(JtJ, False)
    hmin = np.sqrt(np.maximum(lamJ, 0.0)) / order
    with np.errstate(divide="ignore", invalid="ignore"):
        inv_dt = cs / hmin + 2.5 * mu / (rho * hmin * hmin)
    m = float(np.max(inv_dt)) if N else 0.0
    if inverted or not np.isfinite(m):
        dt_est = 0.0
    elif m == 0.0:
        dt_est = float("inf")
    else:
        dt_est = cfl / m
    return D, dt_est, dict(detJ=detJ, rho=rho, p=pres, cs=cs, mu=mu, eps=eps, hmin=hmin, inverted=inverted)
