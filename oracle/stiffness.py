"""Stiffness (diffusion) operator and the discrete Laplacian it serves.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 2.1 says the hyper-viscosity term of the Lagrange phase needs a
"stiffness matrix" operator besides the mass and force matrices; Section 3.3
repeats that an additional operator is applied for it; Section 6 names the
diffusion-integrator kernels used in the artificial-viscosity calculation. The
paper defers the hyper-viscosity model itself to its reference. Reading:
  * on the mesh with H1 node positions x, the scalar stiffness matrix
        S_ij = int grad w_i . grad w_j dx,       S_v = I_d (x) S,
    from dense element matrices with the Lagrange phase's quadrature
        Se_ij = sum_q omega_q detJ (J^-T ghat_i) . (J^-T ghat_j),
    ghat_i the reference gradient of w_i;
  * the discrete Laplacian of an H1 field v (what a hyper-viscosity indicator
    evaluates): lap = -M_x^{-1} S_x v per component, M_x the unit-density mass
    matrix on x; natural boundary conditions (every DOF).

Pins (tests/test_oracle_stiffness.py): S 1 = 0; the unit-square Q1 element
matrix is the textbook one, (1/6)(4 on the diagonal, -1 to edge neighbours, -2
across); a field linear in x has zero rows at interior nodes on jittered meshes
(int grad w_i . a dx = 0 when w_i vanishes on the boundary; the integrand
ghat^T adj(J) a is a polynomial the quadrature integrates exactly); on an affine
mesh with p >= 2, f = |x|^2/2 lies in the space and its interior rows equal
-d int w_i dx; with p >= 3, f = sum_c (x_c^2/2 - x_c^3/3) has zero normal
derivative on the box faces and Delta f = sum_c (1 - 2 x_c) in the space, so the
discrete Laplacian reproduces Delta f at every node.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import jacobians


def _assemble(mesh, Ae: np.ndarray) -> sp.csr_matrix:
    rows = np.repeat(mesh.e2n, mesh.ND1, axis=1).ravel()
    cols = np.tile(mesh.e2n, (1, mesh.ND1)).ravel()
    return sp.coo_matrix((Ae.ravel(), (rows, cols)), shape=(mesh.NH1, mesh.NH1)).tocsr()


def element_stiffness(T, Xe: np.ndarray) -> np.ndarray:
    """Se[e, i, j] = sum_q w_q detJ (J^-T ghat_i) . (J^-T ghat_j) from element node coordinates."""
    J = jacobians(T, Xe)                                   # [NE, Q, c, l] = dx_c / dxi_l
    detJ = np.linalg.det(J)
    if np.any(detJ <= 0.0):
        raise ValueError("inverted element")
    Jinv = np.linalg.inv(J)                                # [NE, Q, l, c]
    phys = np.einsum("eqlc,lqi->eqci", Jinv, T.G, optimize=True)   # physical gradients
    coef = detJ * T.w[None, :]
    return np.einsum("eq,eqci,eqcj->eij", coef, phys, phys, optimize=True)


def element_mass_unit(T, Xe: np.ndarray) -> np.ndarray:
    """Me[e, i, j] = sum_q w_q detJ w_i w_j (unit density) on the element."""
    detJ = np.linalg.det(jacobians(T, Xe))
    return np.einsum("qi,eq,qj->eij", T.B, detJ * T.w[None, :], T.B, optimize=True)


class Stiffness:
    """Stiffness matrix and discrete Laplacian on the mesh at node positions x."""

    def __init__(self, mesh, T, x: np.ndarray):
        Xe = mesh.gather(np.asarray(x, dtype=np.float64))
        self.mesh = mesh
        self.S = _assemble(mesh, element_stiffness(T, Xe))
        self.M = _assemble(mesh, element_mass_unit(T, Xe))

    def mult(self, v: np.ndarray) -> np.ndarray:
        """S_v v, v: [d][N_H1]."""
        return (self.S @ np.asarray(v).T).T

    def laplacian(self, v: np.ndarray) -> np.ndarray:
        """-M_x^{-1} S_x v per component (natural boundary conditions)."""
        lu = spla.splu(self.M.tocsc())
        return np.stack([-lu.solve(self.S @ vc) for vc in np.asarray(v)])
