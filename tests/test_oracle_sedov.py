"""Pins of the oracle's shock workload (Sedov blast) and of the step control with rejection.

Fixed by the problem, not by the oracle's formulas: the deposited internal energy
is exactly E0 and the kinetic energy 0 at t = 0; the energy-conserving scheme keeps
KE + IE = E0 through shocks (direct solves); a rejected attempt is the identity on
the state; the blast is symmetric under any permutation of the axes on a uniform
mesh (the corner at the origin is on all symmetry planes), which a wrong index,
sign or axis anywhere in the viscosity or the step breaks.
"""
import numpy as np
import pytest

from oracle.hydro import SEDOV_E0, Hydro, Params, controlled_step
from paper_2112_07075_b300 import inputs


def _hydro(dim, n, p=2, q1=4):
    return Hydro(Params(dim=dim, n=n, order=p, q1=q1, vertices=inputs.box_vertices(dim, n), gamma=1.4, cfl=0.5))


def _run(hy, attempts):
    x, v, e = hy.initial_state("sedov")
    t, c, rejected = 0.0, 0.0, 0
    for _ in range(attempts):
        before = [a.copy() for a in (x, v, e)]
        x1, v1, e1, info = controlled_step(hy, x, v, e, t, 1.0, c)
        c = info.extra["c"]
        if info.extra["rejected"]:
            rejected += 1
            for a, b in zip((x1, v1, e1), before):             # identity on the state
                assert np.array_equal(np.asarray(a).reshape(b.shape), b)
            assert c < info.dt
        else:
            t += info.dt
        x, v, e = x1, v1, e1
    return x, v, e, t, rejected


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 3)])
def test_sedov_initial_energy(dim, n):
    hy = _hydro(dim, n)
    x, v, e = hy.initial_state("sedov")
    assert hy.kinetic_energy(v) == 0.0
    assert abs(hy.internal_energy(e) - SEDOV_E0) <= 1e-15
    assert np.count_nonzero(e) == e.shape[1]                   # one element only


@pytest.mark.parametrize("dim,n,attempts", [(2, 8, 14), (3, 3, 10)])
def test_sedov_conserves_energy_through_rejections(dim, n, attempts):
    hy = _hydro(dim, n)
    x, v, e, t, rejected = _run(hy, attempts)
    assert rejected >= 1 and t > 0.0
    assert abs(hy.kinetic_energy(v) + hy.internal_energy(e) - SEDOV_E0) <= 1e-12 * SEDOV_E0
    assert hy.kinetic_energy(v) > 1e-3 * SEDOV_E0                 # the blast moved


def test_sedov_is_symmetric_under_axis_swap_2d():
    n, p = 6, 2
    hy = _hydro(2, n, p)
    x, v, e, _, _ = _run(hy, 8)
    N1 = n * p + 1
    g = np.arange(N1 * N1)
    gx, gy = g % N1, g // N1
    swap = gy + N1 * gx
    assert np.max(np.abs(v[0] - v[1][swap])) <= 1e-12 * np.max(np.abs(v))
    assert np.max(np.abs(x[0] - x[1][swap])) <= 1e-14
    el = np.arange(n * n)
    ex, ey = el % n, el // n
    j = np.arange(p * p)
    jx, jy = j % p, j // p
    e_sw = e[(ey + n * ex)[:, None], (jy + p * jx)[None, :]]
    assert np.max(np.abs(e - e_sw)) <= 1e-12 * np.max(np.abs(e))


def test_sedov_is_symmetric_under_axis_cycle_3d():
    n, p = 3, 2
    hy = _hydro(3, n, p)
    x, v, e, _, _ = _run(hy, 6)
    N1 = n * p + 1
    g = np.arange(N1 ** 3)
    gx, gy, gz = g % N1, (g // N1) % N1, g // (N1 * N1)
    cyc = gz + N1 * (gx + N1 * gy)        # (x, y, z) -> (y, z, x)
    for c in range(3):
        assert np.max(np.abs(v[c] - v[(c + 1) % 3][cyc])) <= 1e-12 * np.max(np.abs(v))
