"""Pins for oracle/hydro.py: conservation, rest state, analytic steady solutions."""
import numpy as np
import pytest

from oracle.hydro import Hydro, Params, gresho_velocity, tg_velocity
from paper_2112_07075_b300 import inputs


def _energy(hy, v, e):
    return hy.kinetic_energy(v) + hy.internal_energy(e)


@pytest.mark.parametrize("dim,n,p,jit,src", [(2, 8, 2, 0.0, "tg2d"), (2, 5, 3, 0.1, "none"),
                                              (3, 3, 2, 0.1, "none")])
def test_total_energy_conserved_to_roundoff(dim, n, p, jit, src):
    hy = Hydro(Params(dim=dim, n=n, order=p, q1=2 * p, source=src,
                      vertices=inputs.box_vertices(dim, n, jitter=jit, seed=11)))
    x, v, e = hy.initial_state("taylor_green")
    E0 = _energy(hy, v, e)
    src_total = 0.0
    for _ in range(5):
        x, v, e, info = hy.rk2avg_step(x, v, e, dt=2e-3)
        src_total += info.energy_source
    E1 = _energy(hy, v, e)
    assert abs(E1 - E0 - src_total) < 2e-14 * E0
    assert np.linalg.norm(v) > 0.0


def test_cfl_time_step_and_final_time():
    hy = Hydro(Params(dim=2, n=4, order=2, q1=4, vertices=inputs.box_vertices(2, 4)))
    x, v, e = hy.initial_state("taylor_green")
    t, t_end, dts = 0.0, 0.02, []
    while t < t_end - 1e-14:
        x, v, e, info = hy.rk2avg_step(x, v, e, dt=None, t=t, t_end=t_end)
        assert info.dt <= info.dt_est + 1e-18
        t += info.dt
        dts.append(info.dt)
    assert abs(t - t_end) < 1e-15
    assert dts[-1] <= dts[0]


def test_uniform_state_at_rest_stays_at_rest():
    hy = Hydro(Params(dim=3, n=2, order=2, q1=4, vertices=inputs.box_vertices(3, 2, jitter=0.1, seed=4)))
    x = hy.mesh.x0
    v = np.zeros_like(x)
    e = np.full((hy.mesh.NE, hy.mesh.NL1), 3.0)
    for _ in range(3):
        x1, v, e1, _ = hy.rk2avg_step(x, v, e, dt=1e-3)
    # pressure forces on interior nodes cancel for a uniform state; boundary
    # normal components are constrained, tangential tractions vanish.
    assert np.max(np.abs(v)) < 1e-13


def test_taylor_green_2d_converges_to_steady_solution():
    errs = []
    for n in (4, 8, 16):
        hy = Hydro(Params(dim=2, n=n, order=2, q1=4, source="tg2d", use_viscosity=False,
                          vertices=inputs.box_vertices(2, n)))
        x, v, e = hy.initial_state("taylor_green")
        for _ in range(10):
            x, v, e, _ = hy.rk2avg_step(x, v, e, dt=2e-3)
        ref = np.where(hy.mesh.free, tg_velocity(x), 0.0)
        errs.append(np.linalg.norm(v - ref) / np.linalg.norm(ref))
    assert errs[0] > 2.5 * errs[1] > 2.5 * 2.5 * errs[2] * 0.4
    assert errs[-1] < 2e-4


def test_gresho_error_decreases_under_refinement():
    errs = []
    for n in (8, 16, 32):
        hy = Hydro(Params(dim=2, n=n, order=2, q1=4, use_viscosity=False,
                          vertices=inputs.box_vertices(2, n, -0.5, 0.5)))
        x, v, e = hy.initial_state("gresho")
        for _ in range(10):
            x, v, e, _ = hy.rk2avg_step(x, v, e, dt=1e-3)
        ref = np.where(hy.mesh.free, gresho_velocity(x), 0.0)
        errs.append(np.linalg.norm(v - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > 2.0 * errs[2]
