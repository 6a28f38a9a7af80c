"""GPU parity of every hot-path row against the FP64 oracle, through the C ABI.

Each operation is called on the same seeded inputs on both sides. Per-operation
results must agree to 1e-12 relative (max norm) -- both sides are FP64 and differ
only in summation order; the end state after the configured steps to 1e-11
relative per field (x, v, e), the tolerance the method's parity target states.
"""
import numpy as np
import pytest

from oracle.hydro import Hydro, Params
from paper_2112_07075_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-12
STEP_TOL = 1e-11


def _ctx(dim, n, p, q1, verts, **kw):
    from paper_2112_07075_b300.lh import Context
    return Context(dim, n, verts, p, q1, **kw)


def _hydro(dim, n, p, q1, verts, **kw):
    return Hydro(Params(dim=dim, n=n, order=p, q1=q1, vertices=verts, **kw))


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = max(np.max(np.abs(b)), 1e-300)
    return float(np.max(np.abs(a - b)) / scale)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


# (dim, n, p, q1, jitter): several tiles, ragged element batches, every compiled family
CASES = [(2, 3, 1, 2, 0.1), (2, 5, 2, 4, 0.15), (2, 3, 2, 3, 0.0), (2, 3, 3, 6, 0.1), (2, 2, 4, 8, 0.1),
         (3, 2, 1, 2, 0.1), (3, 3, 2, 4, 0.15), (3, 2, 3, 6, 0.1), (3, 2, 4, 6, 0.1), (3, 1, 4, 8, 0.0)]


def _state(hy, ctx, seed):
    """Perturbed state: each side adds the same seeded perturbation to its own x0."""
    d, nh1 = hy.mesh.dim, hy.mesh.NH1
    h = 1.0 / hy.prm.n
    dx = inputs.uniform(seed, (d, nh1), -0.03 * h / hy.prm.order, 0.03 * h / hy.prm.order)
    v = inputs.uniform(seed + 1, (d, nh1), -1.0, 1.0)
    e = inputs.uniform(seed + 2, (hy.mesh.NE, hy.mesh.NL1), 0.5, 2.0)
    xg, _, _ = ctx.init_state("taylor_green")
    return (hy.mesh.x0 + dx, v, e), (xg + _t(dx), _t(v), _t(e))


@pytest.mark.parametrize("dim,n,p,q1,jit", CASES)
def test_initial_state(dim, n, p, q1, jit):
    V = inputs.box_vertices(dim, n, jitter=jit, seed=3)
    hy, ctx = _hydro(dim, n, p, q1, V), _ctx(dim, n, p, q1, V)
    xo, vo, eo = hy.initial_state("taylor_green")
    xg, vg, eg = ctx.init_state("taylor_green")
    assert _rel(_np(xg), xo) < 1e-15
    assert _rel(_np(vg), vo) < 1e-14
    assert _rel(_np(eg), eo) < OP_TOL


@pytest.mark.parametrize("dim,n,p,q1,jit", CASES)
@pytest.mark.parametrize("visc", [True, False])
def test_qdata_force_and_transpose(dim, n, p, q1, jit, visc):
    V = inputs.box_vertices(dim, n, jitter=jit, seed=4)
    hy, ctx = _hydro(dim, n, p, q1, V, use_viscosity=visc), _ctx(dim, n, p, q1, V, use_viscosity=visc)
    (xo, vo, eo), (xg, vg, eg) = _state(hy, ctx, 100 + n)
    Do, dt_o, _ = hy.qdata(xo, vo, eo)
    dt_g = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.update_qdata(xg, vg, eg, dt_g)
    Dg = torch.zeros((hy.mesh.NE, dim * dim, hy.T.nq), dtype=torch.float64, device="cuda")
    ctx.copy_qdata(Dg)
    Dg = _np(Dg).reshape(hy.mesh.NE, dim, dim, hy.T.nq).transpose(0, 3, 1, 2)
    assert _rel(Dg, Do) < OP_TOL
    assert abs(_np(dt_g)[0] - dt_o) <= 1e-12 * dt_o
    F = hy.force_matrix(Do)
    # F.1
    rhs = ctx.h1_vector()
    ctx.force_mult(None, rhs)
    assert _rel(_np(rhs), (F @ np.ones(hy.mesh.NL2)).reshape(dim, -1)) < OP_TOL
    # F.u for a random L2 field
    u = inputs.uniform(7, (hy.mesh.NE, hy.mesh.NL1), -1.0, 1.0)
    ctx.force_mult(_t(u), rhs)
    assert _rel(_np(rhs), (F @ u.ravel()).reshape(dim, -1)) < OP_TOL
    # F^T v
    w = inputs.uniform(8, (dim, hy.mesh.NH1), -1.0, 1.0)
    out = ctx.l2_vector()
    ctx.force_mult_t(_t(w), out)
    assert _rel(_np(out), (F.T @ w.ravel()).reshape(hy.mesh.NE, -1)) < OP_TOL
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("dim,n,p,q1,jit", CASES)
def test_mass_mult_cg_and_energy_solve(dim, n, p, q1, jit):
    V = inputs.box_vertices(dim, n, jitter=jit, seed=5)
    hy, ctx = _hydro(dim, n, p, q1, V), _ctx(dim, n, p, q1, V)
    u = inputs.uniform(9, (dim, hy.mesh.NH1), -1.0, 1.0)
    y = ctx.h1_vector()
    ctx.mass_mult(_t(u), y)
    assert _rel(_np(y), hy.mass_mult(u)) < OP_TOL
    b = inputs.uniform(10, (dim, hy.mesh.NH1), -1.0, 1.0)
    x = _t(inputs.uniform(11, (dim, hy.mesh.NH1), -1.0, 1.0))     # non-zero initial guess
    info = ctx.new_cg_info()
    ctx.mass_cg(_t(b), x, 1e-13, 2000, info)
    ci = ctx.read_cg_info(info)
    assert ci.status == 0 and ci.rel_res <= 1e-13 and ci.iters > 0
    ref = hy.mass_solve(b)
    assert _rel(_np(x), ref) < 1e-11
    assert np.all(_np(x)[~hy.mesh.free] == 0.0)
    r = inputs.uniform(12, (hy.mesh.NE, hy.mesh.NL1), -1.0, 1.0)
    out = ctx.l2_vector()
    ctx.energy_solve(_t(r), out)
    assert _rel(_np(out), hy.energy_solve(r)) < 1e-11


def test_cg_zero_rhs_and_iteration_limit():
    V = inputs.box_vertices(2, 4)
    ctx = _ctx(2, 4, 2, 4, V)
    x = _t(np.ones((2, ctx.sizes.n_h1)))
    info = ctx.new_cg_info()
    ctx.mass_cg(ctx.h1_vector(), x, 1e-12, 100, info)
    ci = ctx.read_cg_info(info)
    assert ci.status == 0 and ci.iters == 0 and float(_np(x).max()) == 0.0
    b = _t(inputs.uniform(1, (2, ctx.sizes.n_h1)))
    ctx.mass_cg(b, x, 1e-14, 2, info)
    ci = ctx.read_cg_info(info)
    assert ci.status == 5 and ci.iters == 2
    assert ctx.sync_status() == 5          # latched, then cleared
    assert ctx.sync_status() == 0


def _run_steps(dim, n, p, q1, jit, steps, dt, lo=0.0, hi=1.0, problem="taylor_green", source="none", t_end=None):
    V = inputs.box_vertices(dim, n, lo, hi, jitter=jit, seed=6)
    hy = _hydro(dim, n, p, q1, V, source=source)
    ctx = _ctx(dim, n, p, q1, V, source=source)
    xo, vo, eo = hy.initial_state(problem)
    xg, vg, eg = ctx.init_state(problem)
    info = ctx.new_step_info(0.0, t_end if t_end else 0.0)
    t = 0.0
    for _ in range(steps):
        xo, vo, eo, oi = hy.rk2avg_step(xo, vo, eo, dt=dt, t=t, t_end=t_end)
        t += oi.dt
        ctx.rk2avg_step(xg, vg, eg, dt if dt else 0.0, info)
    si = ctx.read_step_info(info)
    return hy, (xo, vo, eo, t, oi), (_np(xg), _np(vg), _np(eg), si)


def _field_err(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_taylor_green_2d_config_steps_match_oracle():
    """2D Taylor-Green 8x8, Q2/Q1, 4x4 Gauss points, fixed dt 1e-3, 20 steps, with the energy source."""
    hy, (xo, vo, eo, t, _), (xg, vg, eg, si) = _run_steps(2, 8, 2, 4, 0.0, 20, 1e-3, source="tg2d")
    assert si.status == 0 and si.steps == 20
    assert abs(si.t - t) < 1e-15
    for a, b in ((xg, xo), (vg, vo), (eg, eo)):
        assert _field_err(a, b) < STEP_TOL
    assert max(si.cg_rel_res) <= 1e-12


@pytest.mark.parametrize("dim,n,p,q1,jit", [(2, 6, 3, 6, 0.1), (3, 3, 2, 4, 0.1), (3, 2, 3, 6, 0.1)])
def test_cfl_controlled_steps_match_oracle(dim, n, p, q1, jit):
    hy, (xo, vo, eo, t, oi), (xg, vg, eg, si) = _run_steps(dim, n, p, q1, jit, 4, None, t_end=1.0)
    assert si.status == 0
    assert abs(si.dt_est - oi.dt_est) <= 1e-12 * oi.dt_est
    assert abs(si.t - t) <= 1e-14
    for a, b in ((xg, xo), (vg, vo), (eg, eo)):
        assert _field_err(a, b) < STEP_TOL


def test_long_horizon_200_cfl_steps_match_oracle():
    """3D Taylor-Green 4^3 Q2/Q1 (jittered), 200 CFL steps (t ~ 0.25): no slow drift of the
    GPU solution away from the oracle; the CG tolerance (1e-12) enters every stage, so
    the bar is 1e-10 per field after this many steps."""
    hy, (xo, vo, eo, t, oi), (xg, vg, eg, si) = _run_steps(3, 4, 2, 4, 0.1, 200, None, t_end=10.0)
    assert si.status == 0 and si.steps == 200
    assert abs(si.t - t) <= 1e-12 * t
    for a, b in ((xg, xo), (vg, vo), (eg, eo)):
        assert _field_err(a, b) < 1e-10


def test_gresho_steps_match_oracle():
    hy, (xo, vo, eo, t, _), (xg, vg, eg, si) = _run_steps(2, 10, 2, 4, 0.0, 5, 1e-3, -0.5, 0.5, "gresho")
    for a, b in ((xg, xo), (vg, vo), (eg, eo)):
        assert _field_err(a, b) < STEP_TOL


def test_energy_conservation_and_determinism():
    V = inputs.box_vertices(3, 3, jitter=0.1, seed=2)
    hy = _hydro(3, 3, 2, 4, V)
    runs = []
    for _ in range(2):
        ctx = _ctx(3, 3, 2, 4, V)
        x, v, e = ctx.init_state()
        info = ctx.new_step_info()
        for _ in range(5):
            ctx.rk2avg_step(x, v, e, 2e-3, info)
        runs.append((_np(x), _np(v), _np(e)))
    for a, b in zip(*runs):
        assert np.array_equal(a, b)                  # bit-identical across runs
    xo, vo, eo = hy.initial_state("taylor_green")
    E0 = hy.kinetic_energy(vo) + hy.internal_energy(eo)
    x, v, e = runs[0]
    E1 = hy.kinetic_energy(v) + hy.internal_energy(e)
    assert abs(E1 - E0) < 1e-11 * E0                 # CG tolerance 1e-12 bounds the drift



@pytest.mark.parametrize("n", [24, 28])
def test_full_size_runs_are_bit_identical(n):
    """Benchmark-size meshes (every solver block sweeps several element batches, the
    grid barriers and block sums run at full width): two runs from the same state
    give bit-identical fields, iteration counts and times."""
    V = inputs.box_vertices(3, n)
    runs = []
    for _ in range(2):
        ctx = _ctx(3, n, 2, 4, V)
        x, v, e = ctx.init_state()
        info = ctx.new_step_info(0.0, 1.0)
        for _ in range(3):
            ctx.rk2avg_step(x, v, e, 0.0, info)
        si = ctx.read_step_info(info)
        assert si.status == 0
        runs.append((_np(x), _np(v), _np(e), si.cg_iters_total, si.t))
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision,n,p,q1", [("fp32_ir", 16, 4, 6), ("bf16tc_ir", 16, 4, 6), ("fp32_ir", 12, 3, 6),
                                              ("fp32_ir", 24, 2, 4)])
def test_precision_forms_are_bit_identical_across_runs(precision, n, p, q1):
    """The precision forms' solvers (several element batches per CTA at p >= 3, a
    software-pipelined gather at p = 4) give bit-identical fields and times from run
    to run."""
    V = inputs.box_vertices(3, n)
    runs = []
    for _ in range(2):
        ctx = _ctx(3, n, p, q1, V, precision=precision)
        x, v, e = ctx.init_state()
        info = ctx.new_step_info(0.0, 1.0)
        for _ in range(3):
            ctx.rk2avg_step(x, v, e, 0.0, info)
        si = ctx.read_step_info(info)
        assert si.status == 0
        runs.append((_np(x), _np(v), _np(e), si.cg_iters_total, si.t))
    for a, b in zip(*runs):
        assert np.array_equal(a, b)

def test_inverted_element_is_reported():
    V = inputs.box_vertices(2, 2)
    ctx = _ctx(2, 2, 1, 2, V)
    x, v, e = ctx.init_state()
    xh = _np(x)
    xh[0, 4] = 1.2                                   # centre node beyond the right face
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.update_qdata(_t(xh), v, e, dt)
    assert float(_np(dt)[0]) == 0.0
    assert ctx.sync_status() == 4


def test_setup_rejects_inverted_mesh_and_unsupported_order():
    from paper_2112_07075_b300.lh import LhError
    V = inputs.box_vertices(2, 2)
    V[4] = [1.5, 0.5]
    with pytest.raises(LhError):
        _ctx(2, 2, 1, 2, V)
    with pytest.raises(LhError):
        _ctx(2, 2, 2, 7, inputs.box_vertices(2, 2))


def test_bounded_grid_wait_times_out_without_fault():
    """A grid-wide wait whose partner block never arrives gives up (~1 s) and reports LH_ERR_TIMEOUT."""
    import ctypes
    from paper_2112_07075_b300 import lh
    st = ctypes.c_int(-1)
    assert lh.load_library().lh_selftest_barrier_timeout(ctypes.byref(st)) == lh.LH_OK
    assert st.value == lh.LH_ERR_TIMEOUT


def test_config2_full_size_one_step_matches_oracle():
    """3D Taylor-Green 24^3, Q2/Q1, 4^3 Gauss points, one CFL (0.5) step from t = 0 -- the benchmarked
    workload at full size and launch configuration -- against the oracle, 1e-11 per field."""
    V = inputs.box_vertices(3, 24)
    hy = _hydro(3, 24, 2, 4, V)
    ctx = _ctx(3, 24, 2, 4, V)
    xo, vo, eo = hy.initial_state("taylor_green")
    xo, vo, eo, oi = hy.rk2avg_step(xo, vo, eo, dt=None, t=0.0, t_end=0.1)
    xg, vg, eg = ctx.init_state("taylor_green")
    info = ctx.new_step_info(0.0, 0.1)
    ctx.rk2avg_step(xg, vg, eg, 0.0, info)
    si = ctx.read_step_info(info)
    assert si.status == 0 and abs(si.dt - oi.dt) <= 1e-12 * oi.dt
    for a, b in ((_np(xg), xo), (_np(vg), vo), (_np(eg), eo)):
        assert _field_err(a, b) < STEP_TOL
