"""Stiffness operator and discrete Laplacian (Sections 2.1, 3.3, 6) on the GPU against the oracle.

S_x u is compared with the oracle's assembled stiffness matrix (per-operation FP64
bar: 1e-12 of the size of the summed terms), the Laplacian with the oracle's
direct solve (1e-11, GPU solve to 1e-13); without the oracle, the Laplacian of a
field with zero normal derivative and its Laplacian in the space must come out
exact; and at the benchmark size (24^3 Q2 Lagrangian mesh) both are checked
against the oracle's assembled operators with a scipy CG solve.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.fem import Tables
from oracle.mesh import Mesh
from oracle.stiffness import Stiffness
from paper_2112_07075_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-12

FAMILIES = [(2, 1, 2, 5), (2, 2, 3, 4), (2, 2, 4, 9), (2, 3, 6, 3), (2, 4, 8, 3),
            (3, 1, 2, 3), (3, 2, 4, 3), (3, 3, 6, 2), (3, 4, 6, 2), (3, 4, 8, 2)]


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _case(dim, p, q1, n, jit=0.12):
    from paper_2112_07075_b300.lh import Context
    V = inputs.box_vertices(dim, n, jitter=jit, seed=5)
    m = Mesh(V, dim, n, p)
    # a moved mesh: the context's own x0 plus a smooth displacement
    x = m.x0 + 0.02 / n * np.sin(2.0 * np.pi * m.x0[::-1])
    return Context(dim, n, V, p, q1), m, x


@pytest.mark.parametrize("dim,p,q1,n", FAMILIES)
def test_stiffness_action_matches_oracle(dim, p, q1, n):
    ctx, m, x = _case(dim, p, q1, n)
    st = Stiffness(m, Tables(dim, p, q1), x)
    u = inputs.uniform(41, (dim, m.NH1), -1.0, 1.0)
    ctx.stiffness_setup(_dev(x))
    y = ctx.h1_vector()
    ctx.stiffness_mult(_dev(u), y)
    ref = st.mult(u)
    scale = (abs(st.S) @ abs(u).T).max()
    assert np.max(np.abs(_np(y) - ref)) <= OP_TOL * scale
    ctx.stiffness_mult(_dev(np.ones((dim, m.NH1))), y)      # S 1 = 0
    assert np.max(np.abs(_np(y))) <= 1e-13 * scale
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("dim,p,q1,n", [(2, 1, 2, 5), (2, 2, 4, 6), (2, 4, 8, 3), (3, 1, 2, 3), (3, 2, 4, 3),
                                        (3, 3, 6, 2), (3, 4, 6, 2)])
def test_laplacian_matches_oracle(dim, p, q1, n):
    ctx, m, x = _case(dim, p, q1, n)
    st = Stiffness(m, Tables(dim, p, q1), x)
    v = inputs.uniform(42, (dim, m.NH1), -1.0, 1.0)
    ref = st.laplacian(v)
    ctx.stiffness_setup(_dev(x))
    lap = ctx.h1_vector()
    info = ctx.new_cg_info()
    ctx.laplacian(_dev(v), lap, rel_tol=1e-13, max_it=5000, info=info)
    ci = ctx.read_cg_info(info)
    assert ci.status == 0 and ci.rel_res <= 1e-13
    assert np.max(np.abs(_np(lap) - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("dim,p,q1,n", [(2, 3, 6, 3), (2, 4, 8, 2), (3, 3, 6, 2), (3, 4, 6, 2)])
def test_laplacian_of_a_neumann_cubic_is_exact_on_gpu(dim, p, q1, n):
    from paper_2112_07075_b300.lh import Context
    m = Mesh(inputs.box_vertices(dim, n), dim, n, p)
    ctx = Context(dim, n, inputs.box_vertices(dim, n), p, q1)
    X = m.x0
    f = np.sum(X ** 2 / 2 - X ** 3 / 3, axis=0)
    ctx.stiffness_setup(_dev(X))
    lap = ctx.h1_vector()
    ctx.laplacian(_dev(np.stack([f] * dim)), lap, rel_tol=1e-14, max_it=5000)
    exact = np.sum(1.0 - 2.0 * X, axis=0)
    assert np.max(np.abs(_np(lap) - exact[None, :])) <= 1e-10


def test_stiffness_errors_are_reported():
    from paper_2112_07075_b300.lh import LH_ERR_ARG, LH_ERR_INVERTED, Context, LhError
    m = Mesh(inputs.box_vertices(2, 4), 2, 4, 2)
    ctx = Context(2, 4, inputs.box_vertices(2, 4), 2, 4)
    u, y = _dev(np.zeros((2, m.NH1))), ctx.h1_vector()
    with pytest.raises(LhError) as ei:             # no setup yet
        ctx.stiffness_mult(u, y)
    assert ei.value.status == LH_ERR_ARG
    with pytest.raises(LhError) as ei:
        ctx.laplacian(u, y)
    assert ei.value.status == LH_ERR_ARG
    x = m.x0.copy()
    x[0, m.N1 * (m.N1 // 2) + m.N1 // 2] += 0.6    # the central node pushed across its elements
    ctx.stiffness_setup(_dev(x))
    assert ctx.sync_status() == LH_ERR_INVERTED
    ctx.stiffness_setup(_dev(m.x0))
    with pytest.raises(LhError) as ei:
        ctx.stiffness_mult(y, y)                   # aliasing
    assert ei.value.status == LH_ERR_ARG
    assert ctx.sync_status() == 0


def test_full_size_lagrangian_mesh():
    """24^3 Q2 Taylor-Green after 40 CFL steps: S_x v and the Laplacian of v on the
    Lagrangian mesh against the oracle's assembled operators (scipy CG on M_x)."""
    from paper_2112_07075_b300.lh import Context
    n, p, q1 = 24, 2, 4
    V = inputs.box_vertices(3, n)
    ctx = Context(3, n, V, p, q1, cfl=0.5)
    x, v, e = ctx.init_state("taylor_green")
    info = ctx.new_step_info(0.0, 1.0)
    for _ in range(40):
        ctx.rk2avg_step(x, v, e, 0.0, info)
    assert ctx.read_step_info(info).status == 0
    ctx.stiffness_setup(x)
    y, lap = ctx.h1_vector(), ctx.h1_vector()
    ctx.stiffness_mult(v, y)
    cinfo = ctx.new_cg_info()
    ctx.laplacian(v, lap, rel_tol=1e-13, info=cinfo)
    assert ctx.read_cg_info(cinfo).status == 0
    xs, vs, ys, laps = _np(x), _np(v), _np(y), _np(lap)

    st = Stiffness(Mesh(V, 3, n, p), Tables(3, p, q1), xs)
    ref = st.mult(vs)
    assert np.max(np.abs(ys - ref)) <= OP_TOL * (abs(st.S) @ abs(vs).T).max()
    Minv = spla.LinearOperator(st.M.shape, matvec=lambda r, d=1.0 / st.M.diagonal(): d * r)
    for c in range(3):
        sol, flag = spla.cg(st.M, -ref[c], rtol=1e-14, maxiter=2000, M=Minv)
        assert flag == 0
        assert np.max(np.abs(laps[c] - sol)) <= 1e-11 * np.max(np.abs(sol))


@pytest.mark.parametrize("precision,dim,p,q1,n", [("fp32_ir", 2, 2, 4, 6), ("fp32_ir", 3, 2, 4, 3),
                                                  ("bf16tc_ir", 3, 4, 6, 3), ("bf16tc_ir", 3, 3, 6, 4)])
def test_laplacian_in_precision_forms_matches_oracle(precision, dim, p, q1, n):
    from paper_2112_07075_b300.lh import Context
    V = inputs.box_vertices(dim, n, jitter=0.12, seed=5)
    m = Mesh(V, dim, n, p)
    x = m.x0 + 0.02 / n * np.sin(2.0 * np.pi * m.x0[::-1])
    ctx = Context(dim, n, V, p, q1, precision=precision)
    v = inputs.uniform(43, (dim, m.NH1), -1.0, 1.0)
    ref = Stiffness(m, Tables(dim, p, q1), x).laplacian(v)
    ctx.stiffness_setup(_dev(x))
    lap = ctx.h1_vector()
    info = ctx.new_cg_info()
    ctx.laplacian(_dev(v), lap, rel_tol=1e-13, max_it=5000, info=info)
    ci = ctx.read_cg_info(info)
    assert ci.status == 0 and ci.rel_res <= 1e-13 and ci.refinements >= 1
    assert np.max(np.abs(_np(lap) - ref)) <= 1e-10 * np.max(np.abs(ref))
