"""Dense element matrices and global full assembly of the mass and force operators.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The multi-dimensional basis tables are formed as explicit Kronecker products of
the 1D tables (Section 3.2, phi_i(q_k) = phi^1d_{i1}(q_k1) phi^1d_{i2}(q_k2)),
so the oracle never uses sum factorization: every operator is a dense element
matrix assembled into a global scipy.sparse matrix (Table 1, first row).

Definitions (readings of Sections 2.1 and 3.3):
  Jacobian      J[c,l](q) = sum_i x_{c,i} dw_i/dxi_l(q)
  mass          M_ij = sum_e sum_q omega_q rho0 detJ0 w_i w_j, M_v = I_d (x) M
                (the element matrix of Section 3.2 with |J| weighted by rho0)
  energy mass   (M_E)_jk = sum_q omega_q rho0 detJ0 phi_j phi_k (per element)
  force         F_{(i,c), j} = sum_q phi_j(q) sum_l dw_i/dxi_l(q) D_q[c,l],
                D_q[c,l] = omega_q detJ_q sum_b sigma_cb(q) (J_q^{-1})_{lb}
                (i.e. F_ij = int sigma : grad(w_i e_c) phi_j dx)

Pins (tests/test_oracle_fem.py): affine elements give h^d times the Kronecker
product of exact 1D mass matrices (computed symbolically with sympy); total mass
1^T M 1 equals rho |Omega|; a brute-force pure-Python element mass matrix on one
element; columns of F sum to zero over the nodes of each component (momentum);
a uniform pressure gives -F.1 equal to the closed-form boundary traction
p * int_face w_i (GLL weights); for v = x (grad v = I) and no viscosity,
F^T v = -d int p phi_j.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .basis import Basis1D


def _kron_all(mats):
    """Kronecker product with the LAST axis fastest-varying in the combined index,
    i.e. mats = [A_x, A_y, A_z] -> kron(A_z, kron(A_y, A_x))."""
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(m, out)
    return out


class Tables:
    """Full (non-factorized) tensor-product tables for one (dim, p, Q1)."""

    def __init__(self, dim: int, p: int, q1: int):
        b = Basis1D(p, q1)
        self.b1 = b
        self.dim = dim
        self.B = _kron_all([b.B] * dim)                      # [Q^d, D1^d]
        self.Bl = _kron_all([b.Bl] * dim)                    # [Q^d, L1^d]
        self.G = np.stack([_kron_all([b.G if a == l else b.B for a in range(dim)])
                           for l in range(dim)])              # [d, Q^d, D1^d]
        self.w = _kron_all([b.wq[None, :]] * dim).ravel()     # [Q^d]
        self.nq = self.B.shape[0]


def jacobians(T: Tables, Xe: np.ndarray) -> np.ndarray:
    """J[e, q, c, l] = sum_i Xe[e, c, i] G[l, q, i] from element node coordinates Xe[e, c, i]."""
    return np.einsum("eci,lqi->eqcl", Xe, T.G, optimize=True)


def ref_gradients(T: Tables, Ue: np.ndarray) -> np.ndarray:
    """Reference gradient of a vector H1 field: dU[e, q, c, l] = sum_i U[e,c,i] dw_i/dxi_l(q)."""
    return np.einsum("eci,lqi->eqcl", Ue, T.G, optimize=True)


def h1_values(T: Tables, Ue: np.ndarray) -> np.ndarray:
    """Values of an element-local vector H1 field at qpoints: [e, q, c]."""
    return np.einsum("eci,qi->eqc", Ue, T.B, optimize=True)


def l2_values(T: Tables, ue: np.ndarray) -> np.ndarray:
    """Values of an element-local L2 field at qpoints: [e, q]."""
    return ue @ T.Bl.T


def assemble_mass(mesh, T: Tables, rho0detJ0: np.ndarray) -> sp.csr_matrix:
    """Scalar global H1 mass matrix M (N_H1 x N_H1) from Me[e] = B^T diag(omega rho0 detJ0) B."""
    coef = rho0detJ0 * T.w[None, :]                                   # [NE, Q]
    Me = np.einsum("qi,eq,qj->eij", T.B, coef, T.B, optimize=True)
    rows = np.repeat(mesh.e2n, mesh.ND1, axis=1).ravel()
    cols = np.tile(mesh.e2n, (1, mesh.ND1)).ravel()
    return sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(mesh.NH1, mesh.NH1)).tocsr()


def energy_mass(T: Tables, rho0detJ0: np.ndarray) -> np.ndarray:
    """Element L2 mass matrices Me[e] (L1^d x L1^d)."""
    coef = rho0detJ0 * T.w[None, :]
    return np.einsum("qj,eq,qk->ejk", T.Bl, coef, T.Bl, optimize=True)


def force_element(T: Tables, D: np.ndarray) -> np.ndarray:
    """Dense element force matrices Fe[e, c, i, j] = sum_q phi_j(q) sum_l dw_i/dxi_l(q) D[e,q,c,l]."""
    S = np.einsum("lqi,eqcl->eciq", T.G, D, optimize=True)                         # sum over l
    return np.einsum("eciq,qj->ecij", S, T.Bl, optimize=True)


def assemble_force(mesh, T: Tables, D: np.ndarray) -> sp.csr_matrix:
    """Global force matrix F: rows = component-major H1 vector DOFs (c*N_H1 + g), cols = L2 DOFs."""
    Fe = force_element(T, D)                                          # [NE, d, ND1, NL1]
    NE, d, nd, nl = Fe.shape
    rows = (np.arange(d)[None, :, None, None] * mesh.NH1
            + mesh.e2n[:, None, :, None]) + np.zeros((1, 1, 1, nl), dtype=np.int64)
    cols = (np.arange(NE)[:, None, None, None] * nl + np.arange(nl)[None, None, None, :]) \
        + np.zeros((1, d, nd, 1), dtype=np.int64)
    return sp.coo_matrix((Fe.ravel(), (rows.ravel(), cols.ravel())),
                         shape=(d * mesh.NH1, mesh.NL2)).tocsr()
