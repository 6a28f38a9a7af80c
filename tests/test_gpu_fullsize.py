"""Full-size workloads of the benchmark against the oracle on sampled outputs.

At 32^3 Q4/Q3 (6^3 Gauss points, jittered) and 48^3 Q3/Q2 the oracle cannot
assemble the global matrices, so it evaluates its element-level definitions
(Section 3.2-3.3 operators: quadrature data D = omega detJ sigma J^-T, the
element force matrices F_e and mass matrices M_e) on sampled elements and
nodes, on the GPU's own state after one benchmarked CFL step. Sampled values
must agree to the per-operation FP64 bar (1e-12 relative to the sampled
values' size). The precision forms are checked at the same full size against
the FP64 GPU path (1e-10 per field, the forms' target).
"""
import numpy as np
import pytest

from oracle.fem import Tables, force_element, jacobians, l2_values, ref_gradients
from oracle.mesh import Mesh
from oracle.qpoint import qdata as oracle_qdata
from paper_2112_07075_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-12
GAMMA = 5.0 / 3.0


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


class _Sampled:
    """The oracle's element-level operators on a structured mesh, without global assembly."""

    def __init__(self, V, n, p, q1):
        self.mesh = Mesh(V, 3, n, p)
        self.T = Tables(3, p, q1)
        self.p = p
        m, T = self.mesh, self.T
        X0e = m.gather(m.x0)
        vol = 0.0
        for s in range(0, m.NE, 4096):   # total volume (for h0) in chunks
            vol += float(np.sum(np.linalg.det(jacobians(T, X0e[s:s + 4096])) * T.w[None, :]))
        self.h0 = (vol / m.NE) ** (1.0 / 3.0) / p
        self.X0e = X0e

    def qdata(self, els, x, v, e):
        m, T = self.mesh, self.T
        Xe, Ve = m.gather(x)[els], m.gather(v)[els]
        J0 = jacobians(T, self.X0e[els])
        J, dV = jacobians(T, Xe), ref_gradients(T, Ve)
        eq = l2_values(T, e.reshape(m.NE, m.NL1)[els])
        ne, Q = J.shape[0], J.shape[1]
        D, _, _ = oracle_qdata(J.reshape(-1, 3, 3), np.linalg.inv(J0).reshape(-1, 3, 3), dV.reshape(-1, 3, 3),
                               eq.ravel(), np.linalg.det(J0).ravel(), np.tile(T.w, ne), gamma=GAMMA, cfl=0.5,
                               order=self.p, h0=self.h0, use_viscosity=True)
        return D.reshape(ne, Q, 3, 3)

    def elements_of(self, g):
        """(element, local node) pairs that contain H1 node g."""
        hit = np.nonzero(self.mesh.e2n == g)
        return list(zip(hit[0], hit[1]))

    def force_one_at(self, g, x, v, e):
        """(F.1) at node g, all components: sum over the elements around g of F_e 1."""
        pairs = self.elements_of(g)
        els = np.array([p[0] for p in pairs])
        Fe = force_element(self.T, self.qdata(els, x, v, e))      # [ne, 3, ND, NL]
        return sum(Fe[k, :, i, :].sum(axis=1) for k, (_, i) in enumerate(pairs))

    def mass_at(self, g, u):
        """(M u) at node g, all components, from the element mass matrices."""
        m, T = self.mesh, self.T
        out = np.zeros(3)
        for el, i in self.elements_of(g):
            J0 = jacobians(T, self.X0e[[el]])[0]
            coef = np.linalg.det(J0) * T.w
            Me_row = (T.B[:, i] * coef) @ T.B                     # row i of B^T diag(coef) B
            out += (u[:, m.e2n[el]] @ Me_row)
        return out


def _sample_nodes(mesh, rng, k):
    N1 = mesh.N1
    corners = [0, N1 - 1, N1 * N1 * N1 - 1, (N1 // 2) + N1 * ((N1 // 2) + N1 * (N1 // 2))]
    return np.concatenate([corners, rng.integers(0, mesh.NH1, size=k)])


@pytest.mark.parametrize("n,p,q1,jit", [(32, 4, 6, 0.15), (48, 3, 6, 0.1)])
def test_full_size_qdata_force_and_mass_match_oracle_on_samples(n, p, q1, jit):
    from paper_2112_07075_b300.lh import Context
    V = inputs.box_vertices(3, n, jitter=jit, seed=3)
    ctx = Context(3, n, V, p, q1, cfl=0.5)
    x, v, e = ctx.init_state("taylor_green")
    info = ctx.new_step_info(0.0, 0.1)
    ctx.rk2avg_step(x, v, e, 0.0, info)                 # the benchmarked step, full size
    assert ctx.read_step_info(info).status == 0
    ctx.update_qdata(x, v, e, None)
    Dg = torch.zeros((ctx.sizes.ne, 9, q1 ** 3), dtype=torch.float64, device="cuda")
    ctx.copy_qdata(Dg)
    f1 = ctx.h1_vector()
    ctx.force_mult(None, f1)
    mx = ctx.h1_vector()
    ctx.mass_mult(x, mx)
    xs, vs, es = _np(x), _np(v), _np(e)
    Dg, f1, mx = _np(Dg), _np(f1), _np(mx)

    orc = _Sampled(V, n, p, q1)
    rng = np.random.default_rng(7)
    els = np.concatenate([[0, orc.mesh.NE - 1], rng.integers(0, orc.mesh.NE, size=6)])
    Do = orc.qdata(els, xs, vs, es)                                   # [k, Q, 3, 3]
    Dgs = Dg[els].reshape(len(els), 3, 3, q1 ** 3).transpose(0, 3, 1, 2)
    assert np.max(np.abs(Dgs - Do)) <= OP_TOL * np.max(np.abs(Do))

    nodes = _sample_nodes(orc.mesh, rng, 8)
    fo = np.array([orc.force_one_at(g, xs, vs, es) for g in nodes])   # [k, 3]
    fg = np.stack([f1[:, g] for g in nodes])
    assert np.max(np.abs(fg - fo)) <= OP_TOL * np.max(np.abs(fo))
    mo = np.array([orc.mass_at(g, xs) for g in nodes])
    mg = np.stack([mx[:, g] for g in nodes])
    assert np.max(np.abs(mg - mo)) <= OP_TOL * np.max(np.abs(mo))


@pytest.mark.parametrize("n,p,q1,jit", [(32, 4, 6, 0.15), (48, 3, 6, 0.1)])
def test_full_size_precision_forms_match_fp64(n, p, q1, jit):
    from paper_2112_07075_b300.lh import Context
    V = inputs.box_vertices(3, n, jitter=jit, seed=3)
    out = {}
    for prec in ("fp64", "fp32_ir", "bf16tc_ir"):
        ctx = Context(3, n, V, p, q1, cfl=0.5, precision=prec)
        x, v, e = ctx.init_state("taylor_green")
        info = ctx.new_step_info(0.0, 0.1)
        for _ in range(2):
            ctx.rk2avg_step(x, v, e, 0.0, info)
        si = ctx.read_step_info(info)
        assert si.status == 0 and max(si.cg_rel_res) <= 1e-12, (prec, si.status, list(si.cg_rel_res))
        out[prec] = (_np(x), _np(v), _np(e))
        ctx.close()
    for prec in ("fp32_ir", "bf16tc_ir"):
        for a, b in zip(out[prec], out["fp64"]):
            assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b), prec
