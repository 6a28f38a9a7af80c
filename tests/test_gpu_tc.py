"""Precision form with the tensor-core inner operator (tcgen05, BF16 hi/lo operands,
FP32 accumulation) against the oracle.

The element operator alone is an approximation of the mass action (BF16 hi/lo
split, FP32 accumulation): it is checked against the oracle's assembled M to the
split's accuracy. The refined solve must reach the FP64 path's residual criterion,
so its solutions and time steps are held to the same bars as the FP32 precision
form: 1e-11 relative on a mass solve, 1e-10 per field after steps.
"""
import numpy as np
import pytest

from oracle.hydro import Hydro, Params
from paper_2112_07075_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# BF16 hi/lo operands (3 products, the lo*lo term dropped) accumulated in FP32: each
# element product is accurate to ~2^-17 relative; 3e-5 on the norm leaves a margin
# and is still two orders below what a plain BF16 operator (~4e-3) would give.
TC_OP_TOL = 3e-5


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# (n, p, q1, jitter): 81 rows (one partial tile), 192 (a full and a half tile),
# 1536 rows (12 tiles), Q4/q6 and Q3/q6
CASES = [(3, 4, 6, 0.15), (4, 4, 6, 0.1), (8, 3, 6, 0.1), (5, 3, 6, 0.1)]


@pytest.mark.parametrize("n,p,q1,jit", CASES)
def test_tensor_core_mass_action_matches_oracle(n, p, q1, jit):
    from paper_2112_07075_b300.lh import Context
    V = inputs.box_vertices(3, n, jitter=jit, seed=21)
    hy = Hydro(Params(dim=3, n=n, order=p, q1=q1, vertices=V))
    ctx = Context(3, n, V, p, q1, precision="bf16tc_ir")
    u = inputs.uniform(22, (3, hy.mesh.NH1), -1.0, 1.0)
    u = np.where(hy.mesh.free, u, 0.0)
    x = torch.from_numpy(u.astype(np.float32)).cuda()
    y = torch.zeros_like(x)
    ctx.mass_mult_tc(x, y)
    ref = hy.mass_mult(u.astype(np.float32).astype(np.float64))
    err = _rel(_np(y).astype(np.float64), ref)
    assert err < TC_OP_TOL, err
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("n,p,q1,jit", CASES[:3])
def test_tensor_core_mass_solve_matches_oracle(n, p, q1, jit):
    from paper_2112_07075_b300.lh import Context
    V = inputs.box_vertices(3, n, jitter=jit, seed=12)
    hy = Hydro(Params(dim=3, n=n, order=p, q1=q1, vertices=V))
    ctx = Context(3, n, V, p, q1, precision="bf16tc_ir")
    b = inputs.uniform(40, (3, hy.mesh.NH1), -1.0, 1.0)
    x = torch.zeros((3, hy.mesh.NH1), dtype=torch.float64, device="cuda")
    info = ctx.new_cg_info()
    ctx.mass_cg(torch.from_numpy(b).cuda(), x, 1e-12, 5000, info)
    ci = ctx.read_cg_info(info)
    assert ci.status == 0 and ci.rel_res <= 1e-12, (ci.status, ci.rel_res, ci.iters, ci.refinements)
    assert _rel(_np(x), hy.mass_solve(b)) < 1e-11
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("n,p,q1,jit,steps", [(3, 4, 6, 0.15, 3), (4, 3, 6, 0.1, 3)])
def test_tensor_core_steps_match_oracle_within_1e10(n, p, q1, jit, steps):
    from paper_2112_07075_b300.lh import Context
    V = inputs.box_vertices(3, n, jitter=jit, seed=3)
    hy = Hydro(Params(dim=3, n=n, order=p, q1=q1, vertices=V))
    ctx = Context(3, n, V, p, q1, precision="bf16tc_ir")
    xo, vo, eo = hy.initial_state("taylor_green")
    xg, vg, eg = ctx.init_state("taylor_green")
    info = ctx.new_step_info(0.0, 1.0)
    t = 0.0
    for _ in range(steps):
        xo, vo, eo, oi = hy.rk2avg_step(xo, vo, eo, dt=None, t=t, t_end=1.0)
        t += oi.dt
        ctx.rk2avg_step(xg, vg, eg, 0.0, info)
    si = ctx.read_step_info(info)
    assert si.status == 0 and max(si.cg_rel_res) <= 1e-12
    for a, b in ((xg, xo), (vg, vo), (eg, eo)):
        assert _rel(_np(a), b) < 1e-10


@pytest.mark.parametrize("dim,p,q1", [(2, 3, 6), (3, 2, 4), (3, 4, 8)])
def test_tensor_core_form_rejects_unsupported_families(dim, p, q1):
    from paper_2112_07075_b300.lh import Context, LhError
    V = inputs.box_vertices(dim, 2)
    with pytest.raises(LhError) as ei:
        Context(dim, 2, V, p, q1, precision="bf16tc_ir")
    assert ei.value.status == 7   # LH_ERR_UNSUPPORTED
