"""Shock workload (Sedov blast) with step control and rejection on the GPU against the oracle.

Per attempt the GPU must take the oracle's decision (accept or reject, both
taken in FP64 on dt_est(S_h) < dt) with the same dt, dt_est and half-step
estimate to the fields' bar (1e-10 relative: each is a maximum over the
qpoints of a function of the state, so it carries the state's rounding
differences); after the run the fields agree to 1e-10 (the
viscosity's linear and quadratic terms are both active behind the shock). A
rejected attempt leaves the GPU state bitwise unchanged, and KE + IE stays E0.
"""
import numpy as np
import pytest

from oracle.hydro import SEDOV_E0, Hydro, Params, controlled_step
from paper_2112_07075_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT_TOL = 1e-10


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim,n,p,q1,jit,attempts,precision",
                         [(2, 8, 2, 4, 0.0, 16, "fp64"), (3, 4, 2, 4, 0.0, 12, "fp64"),
                          (2, 6, 3, 6, 0.1, 12, "fp64"), (3, 3, 3, 6, 0.05, 8, "fp64"),
                          (2, 8, 2, 4, 0.0, 16, "fp32_ir"), (3, 3, 3, 6, 0.05, 8, "bf16tc_ir")])
def test_sedov_controlled_run_matches_oracle(dim, n, p, q1, jit, attempts, precision):
    """The precision forms' solves stop at the same FP64 residual criterion, so their
    decisions and fields are held to the same bars as the FP64 path."""
    from paper_2112_07075_b300.lh import Context
    V = inputs.box_vertices(dim, n, jitter=jit, seed=2)
    hy = Hydro(Params(dim=dim, n=n, order=p, q1=q1, vertices=V, gamma=1.4, cfl=0.5))
    ctx = Context(dim, n, V, p, q1, gamma=1.4, cfl=0.5, precision=precision)
    ctx.set_dt_control(True)
    xo, vo, eo = hy.initial_state("sedov")
    xg, vg, eg = ctx.init_state("sedov")
    assert np.max(np.abs(_np(eg) - eo.reshape(_np(eg).shape))) <= 1e-14 * np.max(eo)
    assert np.max(np.abs(_np(vg))) == 0.0
    info = ctx.new_step_info(0.0, 1.0)
    t, c, rejections = 0.0, 0.0, 0
    for k in range(attempts):
        before = [_np(a).copy() for a in (xg, vg, eg)]
        xo, vo, eo, oi = controlled_step(hy, xo, vo, eo, t, 1.0, c)
        c = oi.extra["c"]
        ctx.rk2avg_step(xg, vg, eg, 0.0, info)
        si = ctx.read_step_info(info)
        assert si.status == 0, (k, si.status)
        assert bool(si.rejected) == oi.extra["rejected"], k
        assert abs(si.dt - oi.dt) <= DT_TOL * oi.dt, k
        assert abs(si.dt_est - oi.dt_est) <= DT_TOL * oi.dt_est, k
        assert abs(si.dt_est_half - oi.extra["dt_est_half"]) <= DT_TOL * oi.extra["dt_est_half"], k
        assert abs(si.dt_ctl - c) <= DT_TOL * abs(c), k
        if si.rejected:
            rejections += 1
            for a, b in zip((xg, vg, eg), before):
                assert np.array_equal(_np(a), b), k
        else:
            t += oi.dt
    si = ctx.read_step_info(info)
    assert rejections >= 1 and si.rejections == rejections and si.steps == attempts - rejections
    assert abs(si.t - t) <= 1e-12 * t
    for a, b in ((xg, xo), (vg, vo), (eg, eo)):
        assert _rel(_np(a).reshape(np.shape(b)), b) < 1e-10
    ve, ee = _np(vg), _np(eg)
    assert abs(hy.kinetic_energy(ve) + hy.internal_energy(ee) - SEDOV_E0) <= 1e-10 * SEDOV_E0


def test_plain_cfl_steps_are_unchanged_without_control():
    """Control off: the same Sedov steps as the oracle's plain CFL step (no rejections)."""
    from paper_2112_07075_b300.lh import Context
    dim, n, p, q1 = 2, 6, 2, 4
    V = inputs.box_vertices(dim, n)
    hy = Hydro(Params(dim=dim, n=n, order=p, q1=q1, vertices=V, gamma=1.4, cfl=0.5))
    ctx = Context(dim, n, V, p, q1, gamma=1.4, cfl=0.5)
    xo, vo, eo = hy.initial_state("sedov")
    xg, vg, eg = ctx.init_state("sedov")
    info = ctx.new_step_info(0.0, 1.0)
    t = 0.0
    for _ in range(6):
        xo, vo, eo, oi = hy.rk2avg_step(xo, vo, eo, dt=None, t=t, t_end=1.0)
        t += oi.dt
        ctx.rk2avg_step(xg, vg, eg, 0.0, info)
    si = ctx.read_step_info(info)
    assert si.rejections == 0 and si.steps == 6 and si.status == 0
    for a, b in ((xg, xo), (vg, vo), (eg, eo)):
        assert _rel(_np(a).reshape(np.shape(b)), b) < 1e-10
