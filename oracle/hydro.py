"""The Lagrange-phase method: problem setup, initial data, energy source,
global mass solve, energy solve and the RK2-average time step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Semi-discrete system (Section 3.3, Eqs. 14-18, single material, eta = 1):
    M_v dv/dt = -F.1,   rho|J| = rho0|J0|,   M_E de/dt = F^T v (+ b),   dx/dt = v.
Reading of the time integrator (the paper names none; its mini-app uses the
energy-conserving two-stage "RK2-average" scheme):
  stage 1 at S_n:   a0 = M_v^{-1}(-F(S_n).1),  vb0 = v_n + dt/2 a0,
                    de0 = M_E^{-1}(F(S_n)^T vb0 + b(S_n)),
                    S_h = (x_n + dt/2 vb0, vb0, e_n + dt/2 de0)
  stage 2 at S_h:   a = M_v^{-1}(-F(S_h).1),   vb = v_n + dt/2 a,
                    de = M_E^{-1}(F(S_h)^T vb + b(S_h))
  final:            v += dt a,  e += dt de,  x += dt vb.
The force data of a stage is computed once at that stage's state and used for
both F.1 and F^T (this makes sum KE + IE change only by dt 1^T b).
Time step: fixed dt, or dt = min(dt_est(S_n), t_end - t) with dt_est from the
stage-1 quadrature data.
Mass solve: v.n = 0 on the box faces; the system is restricted to the free
DOFs and the acceleration is zero on constrained DOFs. Small systems use a
sparse direct factorization, large ones plain CG to 1e-14 relative residual.
Energy source (2D Taylor-Green only): b_j = sum_q omega rho0 detJ0 Q(x_q) phi_j
with Q = (3 pi / 8)(cos 3pi x cos pi y - cos pi x cos 3pi y) at the current
quadrature-point positions.

Shock workload (reading of the Sedov blast, used to exercise the viscosity's
linear term and the step control): rho0 = 1, v0 = 0, internal energy E0 = 0.25
deposited uniformly in the element at the origin corner (e = E0 / its mass, 0
elsewhere); the box faces are the symmetry planes (v.n = 0).
Step control with rejection (controlled_step): the attempt uses
dt = min(c, dt_est(S_n), t_end - t) (c <= 0: no cap); if the CFL estimate at the
half-step state S_h is smaller than dt, the attempt is rejected (state
unchanged) and c = 0.85 dt_est(S_h) (0.5 dt if S_h has an inverted element);
otherwise it is accepted and a finite c grows by 2 %.

Pins (tests/test_oracle_hydro.py): total energy KE + IE - sum dt 1^T b is
conserved to round-off with direct solves; total mass 1^T M 1 is constant;
a uniform state at rest stays exactly at rest; 2D Taylor-Green with source and
no viscosity stays near its steady analytic solution with error decreasing
under refinement; Gresho (steady) likewise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import (Tables, assemble_force, assemble_mass, energy_mass, h1_values,
                  jacobians, l2_values, ref_gradients)
from .mesh import Mesh
from .qpoint import qdata as qpoint_qdata


@dataclass
class Params:
    dim: int
    n: int
    order: int
    q1: int
    vertices: np.ndarray
    gamma: float = 5.0 / 3.0
    cfl: float = 0.5
    use_viscosity: bool = True
    source: str = "none"          # "none" | "tg2d"
    rho0: np.ndarray | None = None  # [NE, Q^d] or None for 1


# --- analytic initial data (problem definitions) -------------------------------
def tg_velocity(X):
    d = X.shape[0]
    x, y = X[0], X[1]
    if d == 2:
        return np.stack([np.sin(np.pi * x) * np.cos(np.pi * y),
                         -np.cos(np.pi * x) * np.sin(np.pi * y)])
    z = X[2]
    return np.stack([np.sin(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z),
                     -np.cos(np.pi * x) * np.sin(np.pi * y) * np.cos(np.pi * z),
                     np.zeros_like(x)])


def tg_pressure(X, rho=1.0):
    if X.shape[0] == 2:
        return 0.25 * rho * (np.cos(2 * np.pi * X[0]) + np.cos(2 * np.pi * X[1])) + 1.0
    return 100.0 + rho / 16.0 * (np.cos(2 * np.pi * X[0]) + np.cos(2 * np.pi * X[1])) \
        * (np.cos(2 * np.pi * X[2]) + 2.0)


def gresho_velocity(X):
    x, y = X[0], X[1]
    r = np.sqrt(x * x + y * y)
    vt = np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    rs = np.where(r > 0, r, 1.0)
    return np.stack([-vt * y / rs, vt * x / rs])


def gresho_pressure(X):
    x, y = X[0], X[1]
    r = np.sqrt(x * x + y * y)
    rs = np.where(r > 0, r, 1.0)
    inner = 5.0 + 12.5 * r * r
    mid = 9.0 - 4.0 * math.log(0.2) + 12.5 * r * r - 20.0 * r + 4.0 * np.log(rs)
    return np.where(r < 0.2, inner, np.where(r < 0.4, mid, 3.0 + 4.0 * math.log(2.0)))


def tg2d_source(X):
    x, y = X[0], X[1]
    return (3.0 * np.pi / 8.0) * (np.cos(3 * np.pi * x) * np.cos(np.pi * y)
                                  - np.cos(np.pi * x) * np.cos(3 * np.pi * y))


PROBLEMS = {
    "taylor_green": (tg_velocity, tg_pressure),
    "gresho": (gresho_velocity, lambda X: gresho_pressure(X)),
    "sedov": (lambda X: np.zeros_like(X), None),   # energy set element-wise below
}
SEDOV_E0 = 0.25


@dataclass
class StepInfo:
    dt: float = 0.0
    dt_est: float = 0.0
    energy_source: float = 0.0
    extra: dict = field(default_factory=dict)


class Hydro:
    """One Lagrangian hydro problem on a structured mesh, fully assembled."""

    def __init__(self, prm: Params, direct_limit: int = 8000):
        self.prm = prm
        d = prm.dim
        self.mesh = Mesh(prm.vertices, d, prm.n, prm.order)
        self.T = Tables(d, prm.order, prm.q1)
        m, T = self.mesh, self.T
        X0e = m.gather(m.x0)
        J0 = jacobians(T, X0e)                                  # [NE, Q, d, d]
        self.detJ0 = np.linalg.det(J0)
        if np.any(self.detJ0 <= 0):
            raise ValueError("inverted element in the initial mesh")
        self.Jinv0 = np.linalg.inv(J0)
        rho0 = np.ones_like(self.detJ0) if prm.rho0 is None else np.asarray(prm.rho0, float)
        self.rho0detJ0 = rho0 * self.detJ0                      # [NE, Q]
        self.M = assemble_mass(m, T, self.rho0detJ0)            # scalar, N_H1 x N_H1
        self.Me = energy_mass(T, self.rho0detJ0)                # [NE, L, L]
        self.Me_inv = np.linalg.inv(self.Me)
        vol = float(np.sum(self.detJ0 * T.w[None, :]))
        self.volume = vol
        self.h0 = (vol / m.NE) ** (1.0 / d) / prm.order
        self._solvers = []
        for c in range(d):
            idx = np.nonzero(m.free[c])[0]
            Mc = self.M[idx][:, idx].tocsc()
            if idx.size <= direct_limit:
                lu = spla.splu(Mc)
                self._solvers.append((idx, "lu", lu))
            else:
                self._solvers.append((idx, "cg", Mc.tocsr()))

    # --- initial state ---------------------------------------------------------
    def initial_state(self, problem: str):
        vel, pres = PROBLEMS[problem]
        m, T = self.mesh, self.T
        x = m.x0.copy()
        v = vel(x)
        v = np.where(m.free, v, 0.0)               # exact BC on constrained DOFs
        if problem == "sedov":                     # E0 in the corner element at the origin
            e = np.zeros((m.NE, m.NL1))
            e[0, :] = SEDOV_E0 / float(np.sum(self.rho0detJ0[0] * T.w))
            return x, v, e
        Xq = h1_values(T, m.gather(x))             # [NE, Q, d]
        Xq_t = np.transpose(Xq, (2, 0, 1))
        rho0 = self.rho0detJ0 / self.detJ0
        eq = pres(Xq_t) / ((self.prm.gamma - 1.0) * rho0)
        rhs = np.einsum("eq,qj->ej", self.rho0detJ0 * T.w[None, :] * eq, T.Bl)
        e = np.einsum("ejk,ek->ej", self.Me_inv, rhs)
        return x, v, e

    # --- operators -------------------------------------------------------------
    def qdata(self, x, v, e):
        m, T, prm = self.mesh, self.T, self.prm
        Xe, Ve = m.gather(x), m.gather(v)
        J = jacobians(T, Xe)
        dV = ref_gradients(T, Ve)
        eq = l2_values(T, e.reshape(m.NE, m.NL1))
        NE, Q, d = J.shape[0], J.shape[1], J.shape[2]
        D, dt_est, extra = qpoint_qdata(
            J.reshape(-1, d, d), self.Jinv0.reshape(-1, d, d), dV.reshape(-1, d, d),
            eq.ravel(), self.rho0detJ0.ravel(), np.tile(T.w, NE),
            gamma=prm.gamma, cfl=prm.cfl, order=prm.order, h0=self.h0,
            use_viscosity=prm.use_viscosity)
        return D.reshape(NE, Q, d, d), dt_est, extra

    def force_matrix(self, D) -> sp.csr_matrix:
        return assemble_force(self.mesh, self.T, D)

    def mass_mult(self, u):
        """M_v u for a [d][N_H1] field (all DOFs, no boundary conditions)."""
        return np.stack([self.M @ u[c] for c in range(u.shape[0])])

    def mass_solve(self, b, tol=1e-14):
        """Solve M_v a = b on the free DOFs; a = 0 on constrained DOFs."""
        a = np.zeros_like(b)
        for c, (idx, kind, S) in enumerate(self._solvers):
            rhs = b[c, idx]
            if kind == "lu":
                a[c, idx] = S.solve(rhs)
            else:
                a[c, idx] = _cg(S, rhs, tol)
        return a

    def energy_source(self, x):
        if self.prm.source != "tg2d":
            return np.zeros((self.mesh.NE, self.mesh.NL1))
        T = self.T
        Xq = np.transpose(h1_values(T, self.mesh.gather(x)), (2, 0, 1))
        Qs = tg2d_source(Xq)
        return np.einsum("eq,qj->ej", self.rho0detJ0 * T.w[None, :] * Qs, T.Bl)

    def energy_solve(self, rhs):
        m = self.mesh
        return np.einsum("ejk,ek->ej", self.Me_inv, rhs.reshape(m.NE, m.NL1))

    # --- energies --------------------------------------------------------------
    def kinetic_energy(self, v):
        return 0.5 * float(sum(v[c] @ (self.M @ v[c]) for c in range(v.shape[0])))

    def internal_energy(self, e):
        m = self.mesh
        return float(np.sum(np.einsum("ejk,ek->ej", self.Me, e.reshape(m.NE, m.NL1))))

    # --- time step -------------------------------------------------------------
    def _stage(self, x, v, e, v_base, dt):
        D, dt_est, extra = self.qdata(x, v, e)
        F = self.force_matrix(D)
        ones = np.ones(self.mesh.NL2)
        rhs = -(F @ ones).reshape(v.shape)
        a = self.mass_solve(rhs)
        vb = v_base + 0.5 * dt * a
        b = self.energy_source(x)
        de = self.energy_solve((F.T @ vb.ravel()).reshape(b.shape) + b)
        return a, vb, de, b, dt_est

    def rk2avg_step(self, x, v, e, dt=None, t=0.0, t_end=None):
        """One RK2-average step. dt=None: dt = min(dt_est(S_n), t_end - t).

        Returns (x, v, e, StepInfo). e is [NE, L1^d].
        """
        e = e.reshape(self.mesh.NE, self.mesh.NL1)
        D, dt_est, _ = self.qdata(x, v, e)
        if dt is None:
            dt = dt_est if t_end is None else min(dt_est, t_end - t)
        if not dt > 0.0:
            raise RuntimeError("non-positive time step (inverted element?)")
        F = self.force_matrix(D)
        ones = np.ones(self.mesh.NL2)
        a0 = self.mass_solve(-(F @ ones).reshape(v.shape))
        vb0 = v + 0.5 * dt * a0
        b0 = self.energy_source(x)
        de0 = self.energy_solve((F.T @ vb0.ravel()).reshape(b0.shape) + b0)
        xh, vh, eh = x + 0.5 * dt * vb0, vb0, e + 0.5 * dt * de0
        a, vb, de, b, _ = self._stage(xh, vh, eh, v, dt)
        info = StepInfo(dt=dt, dt_est=dt_est, energy_source=dt * float(np.sum(b)))
        return x + dt * vb, v + dt * a, e + dt * de, info


def controlled_step(hy, x, v, e, t, t_end, c):
    """One attempt of a CFL step with rejection (see the module docstring).

    Returns (x, v, e, StepInfo) with extra = {rejected, dt_est_half, c}; a
    rejected attempt returns the input state unchanged.
    """
    e = e.reshape(hy.mesh.NE, hy.mesh.NL1)
    D, dt_est, _ = hy.qdata(x, v, e)
    dt = min(dt_est, t_end - t)
    if c > 0.0:
        dt = min(dt, c)
    if not dt > 0.0:
        raise RuntimeError("non-positive time step (inverted element?)")
    F = hy.force_matrix(D)
    a0 = hy.mass_solve(-(F @ np.ones(hy.mesh.NL2)).reshape(v.shape))
    vb0 = v + 0.5 * dt * a0
    b0 = hy.energy_source(x)
    de0 = hy.energy_solve((F.T @ vb0.ravel()).reshape(b0.shape) + b0)
    xh, vh, eh = x + 0.5 * dt * vb0, vb0, e + 0.5 * dt * de0
    a, vb, de, b, dt_half = hy._stage(xh, vh, eh, v, dt)
    if dt_half < dt:
        c_new = 0.85 * dt_half if dt_half > 0.0 else 0.5 * dt
        return x, v, e, StepInfo(dt=dt, dt_est=dt_est,
                                 extra={"rejected": True, "dt_est_half": dt_half, "c": c_new})
    c_new = 1.02 * c if c > 0.0 else c
    info = StepInfo(dt=dt, dt_est=dt_est, energy_source=dt * float(np.sum(b)),
                    extra={"rejected": False, "dt_est_half": dt_half, "c": c_new})
    return x + dt * vb, v + dt * a, e + dt * de, info


def _cg(A, b, tol):
    """Plain conjugate gradients, stop at ||r||_2 <= tol ||b||_2."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bnorm = math.sqrt(float(b @ b))
    if bnorm == 0.0:
        return x
    for _ in range(20 * b.size + 100):
        if math.sqrt(rr) <= tol * bnorm:
            break
        Ap = A @ p
        alpha = rr / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x
