"""Structured quad/hex mesh, H1 node positions, element restriction and boundary masks.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The element restriction is the operator G of the decomposition A = P^T G^T B^T D B G P
(Section 3.1): it maps global H1 node values to element-local node values. The
oracle stores it as an explicit integer table e2n[e, i] built by brute force.

Numbering (also the layout the CUDA path uses, stated here independently):
  vertices   v = vx + (n+1)*(vy + (n+1)*vz)
  elements   e = ex + n*(ey + n*ez)
  H1 nodes   g = gx + N1*(gy + N1*gz),  N1 = n*p + 1, gx = ex*p + ix
  local H1   i = ix + D1*(iy + D1*iz),  D1 = p + 1
  local L2   j = jx + p*(jy + p*jz)
  qpoints    k = kx + Q1*(ky + Q1*kz)
Vector H1 fields are stored component-major, [d][N_H1].

Readings: the reference element is [0, 1]^d; the H1 position field is the
multilinear vertex map of each element evaluated at the GLL nodes; the boundary
condition is v.n = 0 on every face of the box, so on a face normal to axis c the
c-component of velocity is constrained (both components at corners/edges).

Pins (tests/test_oracle_mesh.py): node positions on an unjittered box equal the
closed-form grid; the restriction table agrees with a pure-Python brute-force
coordinate lookup; constrained-DOF counts equal the closed-form face counts.
"""
from __future__ import annotations

import itertools

import numpy as np

from .basis import gll_points


class Mesh:
    def __init__(self, vertices: np.ndarray, dim: int, n: int, p: int):
        V = np.asarray(vertices, dtype=np.float64)
        if V.shape != ((n + 1) ** dim, dim):
            raise ValueError("vertex array has the wrong shape")
        self.dim, self.n, self.p = dim, n, p
        self.V = V
        self.d1 = p + 1
        self.N1 = n * p + 1
        self.NE = n ** dim
        self.NH1 = self.N1 ** dim
        self.ND1 = self.d1 ** dim
        self.NL1 = p ** dim
        self.NL2 = self.NE * self.NL1
        self._build_restriction()
        self._build_nodes()
        self._build_bc()

    # --- element restriction G ------------------------------------------------
    def _build_restriction(self):
        d, n, p, N1, D1 = self.dim, self.n, self.p, self.N1, self.d1
        e2n = np.zeros((self.NE, self.ND1), dtype=np.int64)
        ecoords = np.array(list(itertools.product(range(n), repeat=d)))[:, ::-1]  # (ex, ey[, ez]) x-fastest
        lcoords = np.array(list(itertools.product(range(D1), repeat=d)))[:, ::-1]
        eidx = sum(ecoords[:, a] * n ** a for a in range(d))
        lidx = sum(lcoords[:, a] * D1 ** a for a in range(d))
        for e_row, ec in zip(eidx, ecoords):
            g = ec[None, :] * p + lcoords
            e2n[e_row, lidx] = sum(g[:, a] * N1 ** a for a in range(d))
        self.e2n = e2n
        self.ecoords = np.zeros((self.NE, d), dtype=np.int64)
        self.ecoords[eidx] = ecoords

    # --- H1 node positions (multilinear map at GLL nodes) ---------------------
    def _build_nodes(self):
        d, n, p, N1 = self.dim, self.n, self.p, self.N1
        z = gll_points(p)
        g = np.array(list(itertools.product(range(N1), repeat=d)))[:, ::-1]
        gidx = sum(g[:, a] * N1 ** a for a in range(d))
        X = np.zeros((d, self.NH1))
        e = np.minimum(g // p, n - 1)            # owning element per axis (lowest index)
        xi = z[g - e * p]                         # reference coordinate per axis
        for corner in itertools.product((0, 1), repeat=d):
            w = np.ones(g.shape[0])
            vi = np.zeros(g.shape[0], dtype=np.int64)
            for a in range(d):
                c = corner[a]
                w *= xi[:, a] if c else (1.0 - xi[:, a])
                vi += (e[:, a] + c) * (n + 1) ** a
            X[:, gidx] += w[None, :] * self.V[vi].T
        self.x0 = X

    # --- boundary conditions v.n = 0 ------------------------------------------
    def _build_bc(self):
        d, N1 = self.dim, self.N1
        g = np.array(list(itertools.product(range(N1), repeat=d)))[:, ::-1]
        gidx = sum(g[:, a] * N1 ** a for a in range(d))
        free = np.ones((d, self.NH1), dtype=bool)
        for c in range(d):
            on_face = (g[:, c] == 0) | (g[:, c] == N1 - 1)
            free[c, gidx[on_face]] = False
        self.free = free                     # [d][N_H1]
        self.free_flat = free.ravel()        # component-major DOF mask

    def gather(self, u: np.ndarray) -> np.ndarray:
        """Apply G to a [d][N_H1] (or [N_H1]) field: element-local [NE][d][ND1] (or [NE][ND1])."""
        if u.ndim == 1:
            return u[self.e2n]
        return np.transpose(u[:, self.e2n], (1, 0, 2))
