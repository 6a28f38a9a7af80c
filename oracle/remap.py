"""Velocity remap of the ALE remap phase: M(tau) dv/dtau = K(tau) v.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 3.5 ("Partial Assembly in Remap Phase") poses the momentum remap as the
continuous-Galerkin semi-discrete system M_v dv/dtau = K_v v over a fictitious
interval tau in [0, 1] while the mesh moves from its source positions x0 to the
target positions x1 (dx/dtau = x_{tau=1} - x_{tau=0}); Section 2.3 gives the
continuous equation d(rho v)/dtau = u . grad(rho v) with u the mesh
displacement. Reading (the paper fixes neither the density weighting nor the
pseudo-time integrator):
  * unit density: the velocity itself is advected;
  * on the mesh x(tau) = x0 + tau u, u = x1 - x0 (an H1 field), scalar
        M(tau)_ij = int w_i w_j dx,   K(tau)_ij = int w_i (u . grad w_j) dx,
    with M_v = I_d (x) M and K_v = I_d (x) K, both from dense element matrices
    (quadrature, Jacobians J(tau) of x(tau)) assembled globally;
  * explicit midpoint rule with n equal steps dtau = 1/n:
        k1 = M(tau)^-1 K(tau) v,  v_h = v + dtau/2 k1,
        k2 = M(tau + dtau/2)^-1 K(tau + dtau/2) v_h,  v <- v + dtau k2;
  * optionally the Lagrange phase's v.n = 0 constraint: constrained DOFs keep
    their value (the boundary nodes of x(tau) slide along the box faces).

Pins (tests/test_oracle_remap.py): K 1 = 0; 1^T M(tau) 1 = the box volume at
every tau; zero displacement leaves v unchanged; a field linear in the physical
coordinates is remapped exactly (v(x1) at the target nodes) without the
constraint, since its advection u . grad v lies in the discrete space and the
midpoint rule integrates the resulting linear-in-tau nodal values exactly.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import h1_values, jacobians


def _assemble(mesh, Ae: np.ndarray) -> sp.csr_matrix:
    """Global scalar N_H1 x N_H1 matrix from element matrices Ae[e, i, j]."""
    rows = np.repeat(mesh.e2n, mesh.ND1, axis=1).ravel()
    cols = np.tile(mesh.e2n, (1, mesh.ND1)).ravel()
    return sp.coo_matrix((Ae.ravel(), (rows, cols)), shape=(mesh.NH1, mesh.NH1)).tocsr()


class Remap:
    """Velocity remap from the H1 node positions x0 to x1 (same mesh topology)."""

    def __init__(self, mesh, T, x0: np.ndarray, x1: np.ndarray, constrained: bool = True):
        self.mesh, self.T = mesh, T
        self.x0 = np.asarray(x0, dtype=np.float64)
        self.u = np.asarray(x1, dtype=np.float64) - self.x0
        self.constrained = constrained

    def element_matrices(self, tau: float):
        """Me[e, i, j] = sum_q w_q detJ w_i w_j, Ke[e, i, j] = sum_q w_q detJ w_i (u . grad w_j) at x(tau)."""
        m, T = self.mesh, self.T
        X = self.x0 + tau * self.u
        J = jacobians(T, m.gather(X))                 # [NE, Q, c, l] = dx_c / dxi_l
        detJ = np.linalg.det(J)
        if np.any(detJ <= 0.0):
            raise ValueError("inverted element on the remap path")
        Jinv = np.linalg.inv(J)                       # [NE, Q, l, c] = dxi_l / dx_c
        coef = detJ * T.w[None, :]
        uq = h1_values(T, m.gather(self.u))           # [NE, Q, c]
        a = np.einsum("eqlc,eqc->eql", Jinv, uq)      # u in reference coordinates
        Me = np.einsum("qi,eq,qj->eij", T.B, coef, T.B, optimize=True)
        Ke = np.einsum("qi,eq,eql,lqj->eij", T.B, coef, a, T.G, optimize=True)
        return Me, Ke

    def operators(self, tau: float):
        Me, Ke = self.element_matrices(tau)
        return _assemble(self.mesh, Me), _assemble(self.mesh, Ke)

    def rate(self, tau: float, v: np.ndarray) -> np.ndarray:
        """dv/dtau = M(tau)^-1 K(tau) v per component; 0 on constrained DOFs."""
        M, K = self.operators(tau)
        out = np.zeros_like(v)
        for c in range(v.shape[0]):
            idx = np.nonzero(self.mesh.free[c])[0] if self.constrained else np.arange(v.shape[1])
            rhs = (K @ v[c])[idx]
            Mc = M[idx][:, idx].tocsc()
            out[c, idx] = spla.splu(Mc).solve(rhs)
        return out

    def remap(self, v: np.ndarray, steps: int) -> np.ndarray:
        """Midpoint-rule integration of dv/dtau over [0, 1] in `steps` equal steps."""
        v = np.array(v, dtype=np.float64)
        h = 1.0 / steps
        for k in range(steps):
            tau = k * h
            k1 = self.rate(tau, v)
            vh = v + 0.5 * h * k1
            k2 = self.rate(tau + 0.5 * h, vh)
            v = v + h * k2
        return v
