"""Precision form (FP32 inner PCG under FP64 iterative refinement) against the oracle.

The mixed-precision solve must reach the same FP64 residual criterion as the FP64
path, so its results are held to the FP64 path's bars: 1e-11 relative on a single
mass solve and, after time steps, at most 1e-10 relative per field against the
FP64 oracle (the precision form's stated target).
"""
import numpy as np
import pytest

from oracle.hydro import Hydro, Params
from paper_2112_07075_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim,n,p,q1,jit", [(2, 6, 2, 4, 0.1), (2, 4, 4, 8, 0.1), (3, 3, 2, 4, 0.15),
                                            (3, 2, 4, 6, 0.15), (3, 3, 3, 6, 0.1)])
def test_ir_mass_solve_matches_oracle(dim, n, p, q1, jit):
    from paper_2112_07075_b300.lh import Context
    V = inputs.box_vertices(dim, n, jitter=jit, seed=12)
    hy = Hydro(Params(dim=dim, n=n, order=p, q1=q1, vertices=V))
    ctx = Context(dim, n, V, p, q1, precision="fp32_ir")
    b = inputs.uniform(40, (dim, hy.mesh.NH1), -1.0, 1.0)
    x = torch.zeros((dim, hy.mesh.NH1), dtype=torch.float64, device="cuda")
    info = ctx.new_cg_info()
    ctx.mass_cg(torch.from_numpy(b).cuda(), x, 1e-12, 5000, info)
    ci = ctx.read_cg_info(info)
    assert ci.status == 0 and ci.rel_res <= 1e-12, (ci.status, ci.rel_res, ci.iters)
    assert _rel(_np(x), hy.mass_solve(b)) < 1e-11
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("dim,n,p,q1,jit,steps,dt", [(2, 8, 2, 4, 0.0, 20, 1e-3), (3, 3, 4, 6, 0.15, 3, None),
                                                     (3, 4, 2, 4, 0.0, 4, None)])
def test_ir_steps_match_oracle_within_1e10(dim, n, p, q1, jit, steps, dt):
    from paper_2112_07075_b300.lh import Context
    src = "tg2d" if dim == 2 else "none"
    V = inputs.box_vertices(dim, n, jitter=jit, seed=3)
    hy = Hydro(Params(dim=dim, n=n, order=p, q1=q1, vertices=V, source=src))
    ctx = Context(dim, n, V, p, q1, source=src, precision="fp32_ir")
    xo, vo, eo = hy.initial_state("taylor_green")
    xg, vg, eg = ctx.init_state("taylor_green")
    info = ctx.new_step_info(0.0, 1.0)
    t = 0.0
    for _ in range(steps):
        xo, vo, eo, oi = hy.rk2avg_step(xo, vo, eo, dt=dt, t=t, t_end=1.0)
        t += oi.dt
        ctx.rk2avg_step(xg, vg, eg, dt if dt else 0.0, info)
    si = ctx.read_step_info(info)
    assert si.status == 0 and max(si.cg_rel_res) <= 1e-12
    for a, b in ((xg, xo), (vg, vo), (eg, eo)):
        assert _rel(_np(a), b) < 1e-10
