"""Velocity remap (Section 3.5, M(tau) dv/dtau = K(tau) v) on the GPU against the oracle.

The operators K(tau) v and M(tau) v are compared with the oracle's assembled
matrices (per-operation FP64 bar: 1e-12 of the size of the summed terms); the
remapped velocity with the oracle's direct solves (1e-11 with the GPU solves
run to 1e-13); and, independently of the oracle, a field linear in the
physical coordinates must arrive exactly at the target nodes.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.fem import Tables
from oracle.mesh import Mesh
from oracle.remap import Remap
from paper_2112_07075_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-12
REMAP_TOL = 1e-11

# (dim, p, q1, n): every compiled family; element counts with ragged tails
# (2D p=2: 16 elements per block, 81 elements; 3D p=2: 4 per block, 27 elements)
FAMILIES = [(2, 1, 2, 5), (2, 2, 3, 4), (2, 2, 4, 9), (2, 3, 6, 3), (2, 4, 8, 3),
            (3, 1, 2, 3), (3, 2, 4, 3), (3, 3, 6, 2), (3, 4, 6, 2), (3, 4, 8, 2)]


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _setup(dim, p, q1, n, jit=0.12, seeds=(1, 2)):
    from paper_2112_07075_b300.lh import Context
    V0 = inputs.box_vertices(dim, n, jitter=jit, seed=seeds[0])
    V1 = inputs.box_vertices(dim, n, jitter=jit, seed=seeds[1])
    m0, m1 = Mesh(V0, dim, n, p), Mesh(V1, dim, n, p)
    ctx = Context(dim, n, V0, p, q1)
    return ctx, m0, m1, Tables(dim, p, q1)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


@pytest.mark.parametrize("dim,p,q1,n", FAMILIES)
def test_remap_operators_match_oracle(dim, p, q1, n):
    ctx, m0, m1, T = _setup(dim, p, q1, n)
    R = Remap(m0, T, m0.x0, m1.x0)
    v = inputs.uniform(31, (dim, m0.NH1), -1.0, 1.0)
    x0, x1, vd = _dev(m0.x0), _dev(m1.x0), _dev(v)
    kv, mv = ctx.h1_vector(), ctx.h1_vector()
    for tau in (0.0, 0.37, 1.0):
        M, K = R.operators(tau)
        ctx.remap_apply(x0, x1, tau, vd, kv, mv)
        k_ref, m_ref = (K @ v.T).T, (M @ v.T).T
        k_scale = (abs(K) @ abs(v).T).max()
        m_scale = (abs(M) @ abs(v).T).max()
        assert np.max(np.abs(_np(kv) - k_ref)) <= OP_TOL * k_scale, tau
        assert np.max(np.abs(_np(mv) - m_ref)) <= OP_TOL * m_scale, tau
        # the convection of a constant vanishes
        ctx.remap_apply(x0, x1, tau, _dev(np.ones((dim, m0.NH1))), kv, None)
        assert np.max(np.abs(_np(kv))) <= 1e-13 * k_scale, tau
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("dim,p,q1,n,steps,constrained",
                         [(2, 1, 2, 5, 2, True), (2, 2, 4, 6, 1, True), (2, 3, 6, 3, 3, False),
                          (2, 4, 8, 3, 2, True), (3, 1, 2, 3, 2, False), (3, 2, 4, 3, 2, True),
                          (3, 3, 6, 2, 1, True), (3, 4, 6, 2, 2, False)])
def test_remap_matches_oracle(dim, p, q1, n, steps, constrained):
    ctx, m0, m1, T = _setup(dim, p, q1, n)
    v0 = inputs.uniform(32, (dim, m0.NH1), -1.0, 1.0)
    if constrained:
        v0 = np.where(m0.free, v0, 0.0)
    ref = Remap(m0, T, m0.x0, m1.x0, constrained=constrained).remap(v0, steps)
    vd = _dev(v0)
    info = ctx.new_remap_info()
    ctx.remap_velocity(_dev(m0.x0), _dev(m1.x0), vd, steps, constrained, rel_tol=1e-13, info=info)
    ri = ctx.read_remap_info(info)
    assert ri.status == 0 and ri.solves == 2 * steps and ri.cg_rel_res_max <= 1e-13, (ri.status, ri.solves)
    assert ri.cg_iters_total >= ri.cg_iters_max > 0
    out = _np(vd)
    assert np.max(np.abs(out - ref)) <= REMAP_TOL * np.max(np.abs(ref))
    if constrained:   # constrained DOFs keep their (zero) value exactly
        assert np.all(out[~m0.free] == 0.0)
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("dim,p,q1,n,steps", [(2, 1, 2, 4, 1), (2, 2, 4, 5, 2), (2, 4, 8, 2, 3),
                                              (3, 2, 4, 3, 2), (3, 3, 6, 2, 1)])
def test_linear_field_is_remapped_exactly_on_gpu(dim, p, q1, n, steps):
    ctx, m0, m1, _ = _setup(dim, p, q1, n)
    rng = np.random.default_rng(3)
    A, b = rng.uniform(-1, 1, (dim, dim)), rng.uniform(-1, 1, dim)
    vd = _dev(A @ m0.x0 + b[:, None])
    ctx.remap_velocity(_dev(m0.x0), _dev(m1.x0), vd, steps, constrained=False, rel_tol=1e-14, max_it=5000)
    exact = A @ m1.x0 + b[:, None]
    assert np.max(np.abs(_np(vd) - exact)) <= 1e-11 * np.max(np.abs(exact))
    assert ctx.sync_status() == 0


def test_zero_displacement_leaves_velocity_bitwise_unchanged():
    ctx, m0, _, _ = _setup(3, 2, 4, 3)
    v0 = np.where(m0.free, inputs.uniform(5, (3, m0.NH1), -1.0, 1.0), 0.0)
    vd = _dev(v0)
    info = ctx.new_remap_info()
    ctx.remap_velocity(_dev(m0.x0), _dev(m0.x0), vd, 3, info=info)
    ri = ctx.read_remap_info(info)
    assert ri.status == 0 and ri.solves == 6 and ri.cg_iters_total == 0
    assert np.array_equal(_np(vd), v0)


def test_inverted_target_mesh_is_reported():
    from paper_2112_07075_b300.lh import LH_ERR_INVERTED
    ctx, m0, _, _ = _setup(2, 2, 4, 4, jit=0.0)
    x1 = m0.x0.copy()
    g = m0.N1 * (m0.N1 // 2) + m0.N1 // 2          # the central node
    x1[0, g] += 0.6                                   # pushed across several elements
    vd = _dev(np.zeros((2, m0.NH1)))
    info = ctx.new_remap_info()
    ctx.remap_velocity(_dev(m0.x0), _dev(x1), vd, 1, max_it=50, info=info)
    assert ctx.read_remap_info(info).status == LH_ERR_INVERTED
    assert ctx.sync_status() == LH_ERR_INVERTED
    assert ctx.sync_status() == 0                     # read and cleared


def test_remap_rejects_bad_arguments():
    from paper_2112_07075_b300.lh import LhError
    ctx, m0, m1, _ = _setup(2, 2, 4, 3)
    x0, x1, v = _dev(m0.x0), _dev(m1.x0), _dev(np.zeros((2, m0.NH1)))
    with pytest.raises(LhError) as ei:
        ctx.remap_velocity(x0, x1, v, 0)
    assert ei.value.status == 1
    with pytest.raises(LhError) as ei:
        ctx.remap_velocity(x0, x1, x0, 1)
    assert ei.value.status == 1
    with pytest.raises(LhError) as ei:
        ctx.remap_apply(x0, x1, 0.5, v, v, None)
    assert ei.value.status == 1


def test_remap_after_lagrange_steps_full_size():
    """24^3 Q2 Taylor-Green: remap the velocity from the Lagrangian mesh after 40 CFL
    steps back to the initial mesh, against the oracle's operators with its own
    solver (scipy CG on the free DOFs to 1e-14, the mass matrix being well conditioned)."""
    from paper_2112_07075_b300.lh import Context
    n, p, q1 = 24, 2, 4
    V = inputs.box_vertices(3, n)
    ctx = Context(3, n, V, p, q1, cfl=0.5)
    x, v, e = ctx.init_state("taylor_green")
    x_init = x.clone()
    info = ctx.new_step_info(0.0, 1.0)
    for _ in range(40):
        ctx.rk2avg_step(x, v, e, 0.0, info)
    assert ctx.read_step_info(info).status == 0
    x_lag, v_lag = _np(x), _np(v)
    steps = 2
    rinfo = ctx.new_remap_info()
    ctx.remap_velocity(x, x_init, v, steps, rel_tol=1e-13, info=rinfo)
    ri = ctx.read_remap_info(rinfo)
    assert ri.status == 0 and ri.solves == 2 * steps
    out = _np(v)

    m = Mesh(V, 3, n, p)
    R = Remap(m, Tables(3, p, q1), x_lag, _np(x_init))

    def rate(tau, w):
        M, K = R.operators(tau)
        r = np.zeros_like(w)
        for c in range(3):
            idx = np.nonzero(m.free[c])[0]
            Mc = M[idx][:, idx]
            r[c, idx], flag = spla.cg(Mc, (K @ w[c])[idx], rtol=1e-14, maxiter=2000,
                                      M=spla.LinearOperator(Mc.shape, matvec=lambda y, d=1.0 / Mc.diagonal(): d * y))
            assert flag == 0
        return r

    ref, h = v_lag.copy(), 1.0 / steps
    for k in range(steps):
        k1 = rate(k * h, ref)
        k2 = rate(k * h + 0.5 * h, ref + 0.5 * h * k1)
        ref = ref + h * k2
    assert np.max(np.abs(out - ref)) <= REMAP_TOL * np.max(np.abs(ref))
    assert np.max(np.abs(ref - v_lag)) > 1e-6 * np.max(np.abs(v_lag))   # the remap did something


@pytest.mark.parametrize("precision,dim,p,q1,n,steps,constrained",
                         [("fp32_ir", 2, 2, 4, 6, 2, True), ("fp32_ir", 3, 2, 4, 3, 1, False),
                          ("bf16tc_ir", 3, 4, 6, 3, 1, True), ("bf16tc_ir", 3, 3, 6, 4, 2, False)])
def test_remap_in_precision_forms_matches_oracle(precision, dim, p, q1, n, steps, constrained):
    """The remap's mass solves in the context's precision form reach the FP64 residual
    criterion, so the result is held to the precision forms' field bar (1e-10)."""
    from paper_2112_07075_b300.lh import Context
    V0 = inputs.box_vertices(dim, n, jitter=0.12, seed=1)
    m0 = Mesh(V0, dim, n, p)
    m1 = Mesh(inputs.box_vertices(dim, n, jitter=0.12, seed=2), dim, n, p)
    ctx = Context(dim, n, V0, p, q1, precision=precision)
    v0 = inputs.uniform(33, (dim, m0.NH1), -1.0, 1.0)
    if constrained:
        v0 = np.where(m0.free, v0, 0.0)
    ref = Remap(m0, Tables(dim, p, q1), m0.x0, m1.x0, constrained=constrained).remap(v0, steps)
    vd = _dev(v0)
    info = ctx.new_remap_info()
    ctx.remap_velocity(_dev(m0.x0), _dev(m1.x0), vd, steps, constrained, rel_tol=1e-13, info=info)
    ri = ctx.read_remap_info(info)
    assert ri.status == 0 and ri.solves == 2 * steps and ri.cg_rel_res_max <= 1e-13
    assert np.max(np.abs(_np(vd) - ref)) <= 1e-10 * np.max(np.abs(ref))
    assert ctx.sync_status() == 0
