"""Mesh-optimisation (TMOP) objective, gradient, Hessian and Hessian diagonal.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 2.2 defines the objective
    F(x) = int mu(T(x)) + gamma int ((x - x0) / d(x0))^2,
Section 3.4 its derivatives with respect to the H1 node positions x_{a,i}
(Eqs. 6 and 7, quadrature over the target element: weights w_q det W, target
Jacobian W, reference gradients of w_i mapped by W^-1) and says the Newton solve
is preconditioned with the Hessian's diagonal. Reading (the paper fixes neither
the metric nor the target nor d(x0)):
  * reference element [0,1]^d, physical Jacobian A = dx/dxbar, T = A W^-1;
  * target: the ideal element of equal size, W = h I, h = (|Omega| / NE)^(1/d)
    of the mesh the caller names (any W is accepted here);
  * shape metrics: 2D  mu_2(T)   = |T|^2 / (2 det T) - 1,
                   3D  mu_303(T) = |T|^2 / (3 det(T)^(2/3)) - 1
    (both vanish exactly on scaled rotations);
  * limiting term with a constant displacement limit d and weight gamma,
    integrated with the same target weights: gamma sum_q w_q det W |x - x0|^2(q) / d^2.
First and second metric derivatives are written out from the chain rule with
the cofactor C = d(det T)/dT:
  2D: dmu = T/tau - |T|^2 C / (2 tau^2)
      d2mu[an,bp] = dab dnp / tau - (T_an C_bp + T_bp C_an) / tau^2
                    + |T|^2 C_an C_bp / tau^3 - |T|^2 dC_an/dT_bp / (2 tau^2)
  3D: dmu = (2/3) tau^(-2/3) T - (2/9) |T|^2 tau^(-5/3) C
      d2mu[an,bp] = (2/3) tau^(-2/3) dab dnp - (4/9) tau^(-5/3) (T_an C_bp + T_bp C_an)
                    + (10/27) |T|^2 tau^(-8/3) C_an C_bp - (2/9) |T|^2 tau^(-5/3) dC_an/dT_bp
The gradient (Eq. 6) and the element Hessians (Eq. 7) are formed with explicit
sums over the quadrature points, the Hessian assembled globally; its diagonal and
action are read off the assembled matrix.

Pins (tests/test_oracle_tmop.py): closed-form metric values (0 on identity and
scaled rotations, a stretched element's value by hand); dmu and d2mu against
central differences of mu and dmu; the assembled gradient against central
differences of F and the Hessian action against central differences of the
gradient, on jittered meshes; Hessian symmetry; an ideal (uniform) mesh has a
zero metric term and a zero metric gradient.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from .fem import h1_values, jacobians


def _levi_civita():
    e = np.zeros((3, 3, 3))
    for a, b, c in itertools.permutations(range(3)):
        e[a, b, c] = np.linalg.det(np.eye(3)[[a, b, c]])
    return e


_EPS = _levi_civita()


def cofactor(T: np.ndarray) -> np.ndarray:
    """C = d(det T)/dT (cofactor matrix), T [..., d, d]."""
    d = T.shape[-1]
    if d == 2:
        C = np.empty_like(T)
        C[..., 0, 0], C[..., 0, 1] = T[..., 1, 1], -T[..., 1, 0]
        C[..., 1, 0], C[..., 1, 1] = -T[..., 0, 1], T[..., 0, 0]
        return C
    return 0.5 * np.einsum("abc,npq,...bp,...cq->...an", _EPS, _EPS, T, T)


def dcofactor(T: np.ndarray) -> np.ndarray:
    """dC_an / dT_bp as [..., a, n, b, p]."""
    d = T.shape[-1]
    out = np.zeros(T.shape[:-2] + (d, d, d, d))
    if d == 2:
        for a, n in itertools.product(range(2), repeat=2):
            out[..., a, n, 1 - a, 1 - n] = 1.0 if a == n else -1.0
        return out
    return np.einsum("abc,npq,...cq->...anbp", _EPS, _EPS, T)


def mu(T: np.ndarray) -> np.ndarray:
    d = T.shape[-1]
    n2 = np.sum(T * T, axis=(-2, -1))
    tau = np.linalg.det(T)
    return n2 / (2.0 * tau) - 1.0 if d == 2 else n2 / (3.0 * np.cbrt(tau) ** 2) - 1.0


def dmu(T: np.ndarray) -> np.ndarray:
    d = T.shape[-1]
    n2 = np.sum(T * T, axis=(-2, -1))[..., None, None]
    tau = np.linalg.det(T)[..., None, None]
    C = cofactor(T)
    if d == 2:
        return T / tau - n2 * C / (2.0 * tau ** 2)
    return (2.0 / 3.0) * tau ** (-2.0 / 3.0) * T - (2.0 / 9.0) * n2 * tau ** (-5.0 / 3.0) * C


def d2mu(T: np.ndarray) -> np.ndarray:
    """Second derivatives as [..., a, n, b, p] = d^2 mu / dT_an dT_bp."""
    d = T.shape[-1]
    I = np.eye(d)
    dd = np.einsum("ab,np->anbp", I, I)
    n2 = np.sum(T * T, axis=(-2, -1))[..., None, None, None, None]
    tau = np.linalg.det(T)[..., None, None, None, None]
    C = cofactor(T)
    TC = np.einsum("...an,...bp->...anbp", T, C) + np.einsum("...bp,...an->...anbp", T, C)
    CC = np.einsum("...an,...bp->...anbp", C, C)
    dC = dcofactor(T)
    if d == 2:
        return dd / tau - TC / tau ** 2 + n2 * CC / tau ** 3 - n2 * dC / (2.0 * tau ** 2)
    return ((2.0 / 3.0) * tau ** (-2.0 / 3.0) * dd - (4.0 / 9.0) * tau ** (-5.0 / 3.0) * TC
            + (10.0 / 27.0) * n2 * tau ** (-8.0 / 3.0) * CC - (2.0 / 9.0) * n2 * tau ** (-5.0 / 3.0) * dC)


class Tmop:
    """TMOP functional on a mesh (topology and tables); positions are arguments."""

    def __init__(self, mesh, T, W: np.ndarray, x0: np.ndarray, gamma: float, dlim: float):
        self.mesh, self.T = mesh, T
        self.W = np.asarray(W, dtype=np.float64)
        self.Winv = np.linalg.inv(self.W)
        self.detW = float(np.linalg.det(self.W))
        self.x0 = np.asarray(x0, dtype=np.float64)
        self.lim = gamma / dlim ** 2
        # Phi[q, i, n] = sum_l dw_i/dxbar_l(q) (W^-1)_{ln}
        self.Phi = np.einsum("lqi,ln->qin", T.G, self.Winv)

    def _qdata(self, x):
        m, T = self.mesh, self.T
        A = jacobians(T, m.gather(np.asarray(x, dtype=np.float64)))   # [NE, Q, c, l]
        Tm = A @ self.Winv
        if np.any(np.linalg.det(Tm) <= 0.0):
            raise ValueError("inverted element")
        dx = h1_values(T, m.gather(np.asarray(x) - self.x0))          # [NE, Q, c]
        return Tm, dx

    def objective(self, x) -> float:
        Tm, dx = self._qdata(x)
        wq = self.T.w * self.detW
        return float(np.sum(wq[None, :] * (mu(Tm) + self.lim * np.sum(dx * dx, axis=-1))))

    def gradient(self, x) -> np.ndarray:
        """dF/dx_{a,i} (Eq. 6 plus the limiting term), [d][N_H1]."""
        m, T = self.mesh, self.T
        Tm, dx = self._qdata(x)
        wq = self.T.w * self.detW
        P = dmu(Tm)                                                    # [NE, Q, a, n]
        ge = np.einsum("q,eqan,qin->eai", wq, P, self.Phi, optimize=True)
        ge += 2.0 * self.lim * np.einsum("q,eqa,qi->eai", wq, dx, T.B, optimize=True)
        out = np.zeros((m.dim, m.NH1))
        for a in range(m.dim):
            np.add.at(out[a], m.e2n, ge[:, a, :])
        return out

    def hessian(self, x) -> sp.csr_matrix:
        """d^2F/dx_{b,j} dx_{a,i} (Eq. 7 plus the limiting term), global index a*N_H1 + i."""
        m, T = self.mesh, self.T
        Tm, _ = self._qdata(x)
        wq = self.T.w * self.detW
        H = d2mu(Tm)                                                   # [NE, Q, a, n, b, p]
        He = np.einsum("q,eqanbp,qin,qjp->eaibj", wq, H, self.Phi, self.Phi, optimize=True)
        mass = 2.0 * self.lim * np.einsum("q,qi,qj->ij", wq, T.B, T.B)
        for a in range(m.dim):
            He[:, a, :, a, :] += mass[None]
        d, nd = m.dim, m.ND1
        gidx = (np.arange(d)[None, :, None] * m.NH1 + m.e2n[:, None, :]).reshape(m.NE, d * nd)
        rows = np.repeat(gidx, d * nd, axis=1).ravel()
        cols = np.tile(gidx, (1, d * nd)).ravel()
        n = d * m.NH1
        return sp.coo_matrix((He.reshape(m.NE, -1).ravel(), (rows, cols)), shape=(n, n)).tocsr()

    def hessian_mult(self, x, u) -> np.ndarray:
        return (self.hessian(x) @ np.asarray(u).ravel()).reshape(self.mesh.dim, self.mesh.NH1)

    def hessian_diag(self, x) -> np.ndarray:
        return self.hessian(x).diagonal().reshape(self.mesh.dim, self.mesh.NH1)
