"""The allocation-free mass product (lh_mass_mult_noalloc) against lh_mass_mult.

Some callers cannot call cudaMalloc -- code in a latency-critical loop that must
not take cudaMalloc's implicit device synchronisation, or an application that
owns all device memory through its own pool. lh_mass_mult_noalloc serves them:
it needs no context and keeps its element-vector scratch in a fixed 32 MiB static
device array. These tests call it through the C ABI and check that two calls in a
row give the same y = M_v x as the context-based lh_mass_mult, within the
per-operation tolerance the other GPU tests use; that a later call leaves the
device's free memory unchanged (it allocates nothing); that a small case agrees
with the oracle's assembled mass matrix; and that the binding rejects tensors of
the wrong type or length before anything reaches the C ABI.

The file name makes pytest collect it last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from oracle.fem import Tables, jacobians
from oracle.hydro import Hydro, Params
from oracle.mesh import Mesh
from paper_2112_07075_b300 import inputs, lh

OP_TOL = 1e-12


def _mass_qdata(dim, n, p, q1, V):
    """omega_q * rho0 * detJ0 at every quadrature point, rho0 = 1, [NE][q1^dim]."""
    m = Mesh(V, dim, n, p)
    T = Tables(dim, p, q1)
    return np.linalg.det(jacobians(T, m.gather(m.x0))) * T.w[None, :]


@pytest.mark.gpu
def test_noalloc_mass_mult_matches_context_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    cases = [(3, 4, 2, 4, 0.1), (2, 5, 3, 6, 0.15)]          # a larger 3D mesh, then a smaller 2D one
    for call, (dim, n, p, q1, jit) in enumerate(cases):
        V = inputs.box_vertices(dim, n, jitter=jit, seed=20 + call)
        ctx = lh.Context(dim, n, V, p, q1)
        x = torch.from_numpy(inputs.uniform(30 + call, (dim, ctx.sizes.n_h1))).cuda()
        mq = torch.from_numpy(np.ascontiguousarray(_mass_qdata(dim, n, p, q1, V))).cuda()
        y_ref = ctx.h1_vector()
        ctx.mass_mult(x, y_ref)
        y = torch.full_like(y_ref, float("nan"))
        lh.mass_mult_noalloc(dim, n, p, q1, mq, x, y)
        torch.cuda.synchronize()
        err = float((y - y_ref).abs().max() / y_ref.abs().max())
        assert err < OP_TOL, (call, err)
        # a later call allocates nothing: the device's free memory is unchanged
        free0 = torch.cuda.mem_get_info()[0]
        y2 = torch.full_like(y_ref, float("nan"))
        lh.mass_mult_noalloc(dim, n, p, q1, mq, x, y2)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.equal(y2, y)
        ctx.close()


@pytest.mark.gpu
def test_noalloc_mass_mult_matches_oracle_assembled_mass():
    torch = pytest.importorskip("torch")
    dim, n, p, q1 = 2, 3, 2, 3
    V = inputs.box_vertices(dim, n, jitter=0.15, seed=41)
    hy = Hydro(Params(dim=dim, n=n, order=p, q1=q1, vertices=V))
    u = inputs.uniform(42, (dim, hy.mesh.NH1))
    ref = hy.mass_mult(u)
    mq = torch.from_numpy(np.ascontiguousarray(_mass_qdata(dim, n, p, q1, V))).cuda()
    x = torch.from_numpy(u).cuda()
    y = torch.empty_like(x)
    lh.mass_mult_noalloc(dim, n, p, q1, mq, x, y)
    torch.cuda.synchronize()
    err = float(np.max(np.abs(y.cpu().numpy() - ref)) / np.max(np.abs(ref)))
    assert err < OP_TOL
    with pytest.raises(ValueError):
        lh.mass_mult_noalloc(dim, n, p, q1, mq.float(), x, y)
    with pytest.raises(ValueError):
        lh.mass_mult_noalloc(dim, n, p, q1, mq, x[:, :-1].contiguous(), y)
    with pytest.raises(ValueError):
        lh.mass_mult_noalloc(dim, n, p, q1, mq[:-1], x, y)


def test_noalloc_rejects_meshes_beyond_the_static_scratch():
    lib = lh.load_library()
    fake = ctypes.c_void_p(256)   # never dereferenced: the size check rejects the call first
    st = lib.lh_mass_mult_noalloc(3, 64, 64, 64, 4, 8, fake, fake, ctypes.c_void_p(512), None)
    assert st == lh.LH_ERR_ARG
    msg = lib.lh_last_error(None).decode()
    assert "32 MiB" in msg and "bytes" in msg
    assert lib.lh_mass_mult_noalloc(4, 2, 2, 2, 2, 4, fake, fake, ctypes.c_void_p(512), None) == lh.LH_ERR_ARG
