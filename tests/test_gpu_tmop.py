"""TMOP kernels (Section 2.2 objective, Section 3.4 Eqs. 6-7, Jacobi diagonal) on the GPU
against the oracle.

Objective, gradient, Hessian action and Hessian diagonal are compared with the
oracle's explicit sums and assembled Hessian (FP64 per-operation bar: 1e-12 of
the size of the summed terms for the Hessian products and diagonal, 1e-11 of the
largest entry for the gradient, whose terms partly cancel), on jittered meshes
for every compiled family, with and without the limiting term; and at the
benchmark size (24^3 Q2 Lagrangian mesh) on sampled nodes.
"""
import numpy as np
import pytest

from oracle.fem import Tables, h1_values, jacobians
from oracle.mesh import Mesh
from oracle.tmop import Tmop, d2mu
from paper_2112_07075_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FAMILIES = [(2, 1, 2, 5), (2, 2, 3, 4), (2, 2, 4, 6), (2, 3, 6, 3), (2, 4, 8, 3),
            (3, 1, 2, 3), (3, 2, 4, 3), (3, 3, 6, 2), (3, 4, 6, 2), (3, 4, 8, 2)]


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _case(dim, p, q1, n, gamma):
    from paper_2112_07075_b300.lh import Context
    V = inputs.box_vertices(dim, n, jitter=0.15, seed=7)
    m = Mesh(V, dim, n, p)
    x0 = Mesh(inputs.box_vertices(dim, n), dim, n, p).x0
    h = 1.0 / n
    tm = Tmop(m, Tables(dim, p, q1), h * np.eye(dim), x0, gamma=gamma, dlim=0.5 * h)
    return Context(dim, n, V, p, q1), m, tm, x0, h


@pytest.mark.parametrize("gamma", [0.0, 0.3])
@pytest.mark.parametrize("dim,p,q1,n", FAMILIES)
def test_tmop_kernels_match_oracle(dim, p, q1, n, gamma):
    ctx, m, tm, x0, h = _case(dim, p, q1, n, gamma)
    x = m.x0
    kw = dict(h=h, gamma=gamma, dlim=0.5 * h)
    xd, x0d = _dev(x), _dev(x0)
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.tmop_objective(xd, x0d if gamma else None, F, **kw)
    Fo = tm.objective(x)
    assert abs(float(_np(F)[0]) - Fo) <= 1e-12 * abs(Fo)

    g = ctx.h1_vector()
    ctx.tmop_gradient(xd, x0d if gamma else None, g, **kw)
    go = tm.gradient(x)
    assert np.max(np.abs(_np(g) - go)) <= 1e-11 * np.max(np.abs(go))

    H = tm.hessian(x)
    u = inputs.uniform(51, (dim, m.NH1), -1.0, 1.0)
    y = ctx.h1_vector()
    ctx.tmop_hessian_mult(xd, _dev(u), y, **kw)
    ref = (H @ u.ravel()).reshape(dim, m.NH1)
    scale = (abs(H) @ abs(u).ravel()).max()
    assert np.max(np.abs(_np(y) - ref)) <= 1e-12 * scale

    dg = ctx.h1_vector()
    ctx.tmop_hessian_diag(xd, dg, **kw)
    do = H.diagonal().reshape(dim, m.NH1)
    assert np.max(np.abs(_np(dg) - do)) <= 1e-12 * np.max(np.abs(do))
    assert ctx.sync_status() == 0


def test_ideal_mesh_gives_zero_metric_and_gradient_on_gpu():
    from paper_2112_07075_b300.lh import Context
    n, p, q1 = 4, 2, 4
    V = inputs.box_vertices(3, n)
    ctx = Context(3, n, V, p, q1)
    x = _dev(Mesh(V, 3, n, p).x0)
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.tmop_objective(x, None, F, h=1.0 / n)
    g = ctx.h1_vector()
    ctx.tmop_gradient(x, None, g, h=1.0 / n)
    assert abs(float(_np(F)[0])) < 1e-13
    assert np.max(np.abs(_np(g))) < 1e-13


def test_tmop_errors_are_reported():
    from paper_2112_07075_b300.lh import LH_ERR_ARG, LH_ERR_INVERTED, Context, LhError
    n = 4
    V = inputs.box_vertices(2, n)
    m = Mesh(V, 2, n, 2)
    ctx = Context(2, n, V, 2, 4)
    x = _dev(m.x0)
    g = ctx.h1_vector()
    with pytest.raises(LhError) as ei:              # limiting term without x0
        ctx.tmop_gradient(x, None, g, h=0.25, gamma=1.0, dlim=0.1)
    assert ei.value.status == LH_ERR_ARG
    with pytest.raises(LhError) as ei:              # bad target size
        ctx.tmop_gradient(x, None, g, h=0.0)
    assert ei.value.status == LH_ERR_ARG
    with pytest.raises(LhError) as ei:              # aliasing
        ctx.tmop_hessian_mult(x, g, g, h=0.25)
    assert ei.value.status == LH_ERR_ARG
    xi = m.x0.copy()
    xi[0, m.N1 * (m.N1 // 2) + m.N1 // 2] += 0.6     # central node pushed across its elements
    ctx.tmop_hessian_diag(_dev(xi), g, h=0.25)
    assert ctx.sync_status() == LH_ERR_INVERTED


def test_full_size_lagrangian_mesh_on_samples():
    """24^3 Q2 Taylor-Green after 40 CFL steps (x0 = the initial mesh for the limiting
    term): objective and gradient against the oracle everywhere, Hessian action and
    diagonal on sampled nodes from the oracle's element Hessians (Eq. 7)."""
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
    h, gamma, dlim = 1.0 / n, 0.1, 0.5 / n
    kw = dict(h=h, gamma=gamma, dlim=dlim)
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    g, y, dg = ctx.h1_vector(), ctx.h1_vector(), ctx.h1_vector()
    u = _dev(inputs.uniform(52, (3, ctx.sizes.n_h1), -1.0, 1.0))
    ctx.tmop_objective(x, x_init, F, **kw)
    ctx.tmop_gradient(x, x_init, g, **kw)
    ctx.tmop_hessian_mult(x, u, y, **kw)
    ctx.tmop_hessian_diag(x, dg, **kw)
    assert ctx.sync_status() == 0
    xs, x0s, us = _np(x), _np(x_init), _np(u)
    Fg, gg, yg, dgg = float(_np(F)[0]), _np(g), _np(y), _np(dg)

    m = Mesh(V, 3, n, p)
    T = Tables(3, p, q1)
    tm = Tmop(m, T, h * np.eye(3), x0s, gamma=gamma, dlim=dlim)
    Fo = tm.objective(xs)
    assert abs(Fg - Fo) <= 1e-12 * abs(Fo)
    go = tm.gradient(xs)
    assert np.max(np.abs(gg - go)) <= 1e-11 * np.max(np.abs(go))

    rng = np.random.default_rng(9)
    nodes = np.concatenate([[0, m.NH1 - 1, m.NH1 // 2], rng.integers(0, m.NH1, size=8)])
    wq = T.w * h ** 3
    Phi = T.G.transpose(1, 2, 0) / h                      # [q, i, n]
    mass = 2.0 * (gamma / dlim ** 2) * np.einsum("q,qi,qj->ij", wq, T.B, T.B)
    for gnode in nodes:
        els, loc = np.nonzero(m.e2n == gnode)
        Xe = m.gather(xs)[els]
        A = jacobians(T, Xe)                              # [k, q, c, l]
        Hq = d2mu(A / h)                                  # [k, q, a, n, b, p]
        Hu, Hd = np.zeros(3), np.zeros(3)
        for k, (el, i) in enumerate(zip(els, loc)):
            Ue = us[:, m.e2n[el]]                         # [b, j]
            # row (a, i) of the element Hessian applied to u_e
            t = np.einsum("q,qanbp,qn,qjp,bj->a", wq, Hq[k], Phi[:, i, :], Phi, Ue)
            Hu += t + mass[i] @ Ue.T
            Hd += np.einsum("q,qanap,qn,qp->a", wq, Hq[k], Phi[:, i, :], Phi[:, i, :]) + mass[i, i]
        scale = max(np.max(np.abs(Hu)), 1e-30)
        assert np.max(np.abs(yg[:, gnode] - Hu)) <= 1e-10 * max(scale, np.max(np.abs(yg))), gnode
        assert np.max(np.abs(dgg[:, gnode] - Hd)) <= 1e-12 * np.max(np.abs(Hd)), gnode


@pytest.mark.parametrize("dim,p,q1,n", FAMILIES)
def test_partially_assembled_hessian_matches_oracle(dim, p, q1, n):
    ctx, m, tm, x0, h = _case(dim, p, q1, n, 0.3)
    x = m.x0
    kw = dict(h=h, gamma=0.3, dlim=0.5 * h)
    work = ctx.tmop_workspace()
    assert work.numel() == m.NE * (dim * dim) * (dim * dim + 1) // 2 * q1 ** dim
    ctx.tmop_hessian_setup(_dev(x), work, **kw)
    H = tm.hessian(x)
    for seed in (61, 62):                     # several products from one setup
        u = inputs.uniform(seed, (dim, m.NH1), -1.0, 1.0)
        y, ymf = ctx.h1_vector(), ctx.h1_vector()
        ctx.tmop_hessian_mult_pa(work, _dev(u), y, **kw)
        ctx.tmop_hessian_mult(_dev(x), _dev(u), ymf, **kw)
        ref = (H @ u.ravel()).reshape(dim, m.NH1)
        scale = (abs(H) @ abs(u).ravel()).max()
        assert np.max(np.abs(_np(y) - ref)) <= 1e-12 * scale
        assert np.max(np.abs(_np(y) - _np(ymf))) <= 1e-12 * scale
    assert ctx.sync_status() == 0
