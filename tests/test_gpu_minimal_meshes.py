"""Degenerate sizes of the widened operators: a single element (n = 1) in 2D and 3D,
where every node is a boundary node and every copy count is one, against the oracle.
"""
import numpy as np
import pytest

from oracle.fem import Tables
from oracle.mesh import Mesh
from oracle.remap import Remap
from oracle.stiffness import Stiffness
from oracle.tmop import Tmop
from paper_2112_07075_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("dim,p,q1", [(2, 1, 2), (2, 4, 8), (3, 2, 4), (3, 4, 6)])
def test_single_element_operators(dim, p, q1):
    from paper_2112_07075_b300.lh import Context
    V = inputs.box_vertices(dim, 1)
    m = Mesh(V, dim, 1, p)
    T = Tables(dim, p, q1)
    ctx = Context(dim, 1, V, p, q1)
    rng = np.random.default_rng(4)
    x1 = m.x0 + 0.05 * rng.uniform(-1, 1, m.x0.shape)      # a skewed target element
    v = inputs.uniform(6, (dim, m.NH1), -1.0, 1.0)
    # remap operators and an unconstrained remap
    kv, mv = ctx.h1_vector(), ctx.h1_vector()
    ctx.remap_apply(_dev(m.x0), _dev(x1), 0.5, _dev(v), kv, mv)
    M, K = Remap(m, T, m.x0, x1).operators(0.5)
    assert np.max(np.abs(_np(kv) - (K @ v.T).T)) <= 1e-12 * (abs(K) @ abs(v).T).max()
    assert np.max(np.abs(_np(mv) - (M @ v.T).T)) <= 1e-12 * (abs(M) @ abs(v).T).max()
    vd = _dev(v)
    ctx.remap_velocity(_dev(m.x0), _dev(x1), vd, 2, constrained=False, rel_tol=1e-14, max_it=2000)
    ref = Remap(m, T, m.x0, x1, constrained=False).remap(v, 2)
    assert np.max(np.abs(_np(vd) - ref)) <= 1e-11 * np.max(np.abs(ref))
    # stiffness and Laplacian
    st = Stiffness(m, T, x1)
    ctx.stiffness_setup(_dev(x1))
    y = ctx.h1_vector()
    ctx.stiffness_mult(_dev(v), y)
    assert np.max(np.abs(_np(y) - st.mult(v))) <= 1e-12 * (abs(st.S) @ abs(v).T).max()
    lap = ctx.h1_vector()
    ctx.laplacian(_dev(v), lap, rel_tol=1e-14, max_it=2000)
    lref = st.laplacian(v)
    assert np.max(np.abs(_np(lap) - lref)) <= 1e-11 * np.max(np.abs(lref))
    # TMOP gradient and Hessian diagonal
    tm = Tmop(m, T, np.eye(dim), m.x0, gamma=0.2, dlim=0.5)
    g, dg = ctx.h1_vector(), ctx.h1_vector()
    ctx.tmop_gradient(_dev(x1), _dev(m.x0), g, h=1.0, gamma=0.2, dlim=0.5)
    go = tm.gradient(x1)
    assert np.max(np.abs(_np(g) - go)) <= 1e-11 * np.max(np.abs(go))
    ctx.tmop_hessian_diag(_dev(x1), dg, h=1.0, gamma=0.2, dlim=0.5)
    do = tm.hessian_diag(x1)
    assert np.max(np.abs(_np(dg) - do)) <= 1e-12 * np.max(np.abs(do))
    assert ctx.sync_status() == 0
