"""Thin ctypes binding of liblh.so (include/lh.h) with the same names.

Argument marshalling only: device buffers are torch CUDA tensors whose raw
pointers are passed to the library; every step of the hot path runs in the
library's CUDA kernels. The library is loaded from this package directory; if it
is missing the import fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblh.so")

LH_OK, LH_ERR_ARG, LH_ERR_CUDA, LH_ERR_OOM, LH_ERR_INVERTED, LH_ERR_NOT_CONVERGED, LH_ERR_TIMEOUT, \
    LH_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["ok", "argument", "cuda", "out of memory", "inverted", "not converged", "timeout", "unsupported"]
PROBLEMS = {"taylor_green": 0, "gresho": 1, "sedov": 2}
SOURCES = {"none": 0, "tg2d": 1}
PRECISIONS = {"fp64": 0, "fp32_ir": 1, "bf16tc_ir": 2}

EXPORTED = ["lh_setup", "lh_destroy", "lh_get_sizes", "lh_last_error", "lh_sync_status", "lh_init_state",
            "lh_update_qdata", "lh_copy_qdata", "lh_force_mult", "lh_force_mult_t", "lh_mass_mult",
            "lh_mass_cg", "lh_energy_solve", "lh_rk2avg_step", "lh_mass_mult_noalloc",
            "lh_batch_create", "lh_batch_autotune", "lh_batch_set_config", "lh_batch_step", "lh_batch_last_error",
            "lh_batch_destroy",
            "lh_mlp_create", "lh_mlp_destroy", "lh_mlp_num_params", "lh_mlp_get_params", "lh_mlp_set_params",
            "lh_mlp_forward", "lh_mlp_gradients", "lh_mlp_train_step", "lh_mlp_last_error", "lh_mlp_sync_status",
            "lh_learn_attach", "lh_learn_set_record_stride",
            "lh_learn_stats", "lh_selftest_barrier_timeout", "lh_timing_enable", "lh_timing_read", "lh_mass_mult_tc",
            "lh_remap_velocity", "lh_remap_apply", "lh_stiffness_setup", "lh_stiffness_mult", "lh_laplacian",
            "lh_tmop_objective", "lh_tmop_gradient", "lh_tmop_hessian_mult", "lh_tmop_hessian_diag",
            "lh_set_dt_control", "lh_tmop_workspace_size", "lh_tmop_hessian_setup", "lh_tmop_hessian_mult_pa"]


class LhParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("vertices", ctypes.POINTER(ctypes.c_double)), ("order", ctypes.c_int), ("q1", ctypes.c_int),
                ("gamma", ctypes.c_double), ("cfl", ctypes.c_double), ("use_viscosity", ctypes.c_int),
                ("source", ctypes.c_int), ("precision", ctypes.c_int)]


class LhSizes(ctypes.Structure):
    _fields_ = [("ne", ctypes.c_int64), ("n_h1", ctypes.c_int64), ("nv", ctypes.c_int64),
                ("n_l2", ctypes.c_int64), ("nq", ctypes.c_int64), ("arena_bytes", ctypes.c_int64)]


class LhCgInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("b_norm", ctypes.c_double), ("refinements", ctypes.c_int), ("reserved", ctypes.c_int)]


class LhStepInfo(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("t_end", ctypes.c_double), ("dt", ctypes.c_double),
                ("dt_est", ctypes.c_double), ("energy_src", ctypes.c_double),
                ("cg_rel_res", ctypes.c_double * 2), ("cg_iters", ctypes.c_int * 2),
                ("status", ctypes.c_int), ("steps", ctypes.c_int), ("cg_iters_total", ctypes.c_longlong),
                ("dt_ctl", ctypes.c_double), ("dt_est_half", ctypes.c_double), ("rejected", ctypes.c_int),
                ("rejections", ctypes.c_int)]


class LhTmopParams(ctypes.Structure):
    _fields_ = [("target_size", ctypes.c_double), ("lim_weight", ctypes.c_double), ("lim_dist", ctypes.c_double)]


class LhRemapInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("solves", ctypes.c_int), ("cg_iters_max", ctypes.c_int),
                ("reserved", ctypes.c_int), ("cg_iters_total", ctypes.c_longlong),
                ("cg_rel_res_max", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblh.so (once). Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"liblh.so not found at {path}; build it with python -m paper_2112_07075_b300.build")
    lib = ctypes.CDLL(path)
    P, I, D, VP = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "lh_setup": (I, [ctypes.POINTER(LhParams), P, ctypes.POINTER(P)]),
        "lh_destroy": (None, [P]),
        "lh_get_sizes": (I, [P, ctypes.POINTER(LhSizes)]),
        "lh_last_error": (ctypes.c_char_p, [P]),
        "lh_sync_status": (I, [P]),
        "lh_init_state": (I, [P, I, VP, VP, VP, VP]),
        "lh_update_qdata": (I, [P, VP, VP, VP, VP, VP]),
        "lh_copy_qdata": (I, [P, VP, VP]),
        "lh_force_mult": (I, [P, VP, VP, VP]),
        "lh_force_mult_t": (I, [P, VP, VP, VP]),
        "lh_mass_mult": (I, [P, VP, VP, VP]),
        "lh_mass_cg": (I, [P, VP, VP, D, I, VP, VP]),
        "lh_energy_solve": (I, [P, VP, VP, VP]),
        "lh_rk2avg_step": (I, [P, VP, VP, VP, D, D, I, VP, VP]),
        "lh_mass_mult_noalloc": (I, [I, I, I, I, I, I, VP, VP, VP, VP]),
        "lh_batch_create": (I, [I, ctypes.POINTER(P), ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.POINTER(VP),
                                ctypes.POINTER(D), VP, ctypes.POINTER(P)]),
        "lh_batch_autotune": (I, [P, ctypes.POINTER(I)]),
        "lh_batch_set_config": (I, [P, ctypes.POINTER(I)]),
        "lh_batch_step": (I, [P, D, I, VP]),
        "lh_batch_last_error": (ctypes.c_char_p, [P]),
        "lh_batch_destroy": (None, [P]),
        "lh_mlp_create": (I, [ctypes.c_ulonglong, I, ctypes.POINTER(P)]),
        "lh_mlp_destroy": (None, [P]),
        "lh_mlp_num_params": (I, []),
        "lh_mlp_get_params": (I, [P, VP]),
        "lh_mlp_set_params": (I, [P, VP]),
        "lh_mlp_forward": (I, [P, VP, I, VP, VP]),
        "lh_mlp_gradients": (I, [P, VP, VP, I, VP, VP, VP]),
        "lh_mlp_train_step": (I, [P, VP, VP, I, ctypes.c_float, VP, VP]),
        "lh_mlp_last_error": (ctypes.c_char_p, [P]),
        "lh_mlp_sync_status": (I, [P]),
        "lh_learn_attach": (I, [P, P, I, VP, VP, I]),
        "lh_learn_set_record_stride": (I, [P, I]),
        "lh_selftest_barrier_timeout": (I, [ctypes.POINTER(I)]),
        "lh_timing_enable": (I, [P, I]),
        "lh_set_dt_control": (I, [P, I]),
        "lh_mass_mult_tc": (I, [P, VP, VP, VP]),
        "lh_remap_velocity": (I, [P, VP, VP, VP, I, I, D, I, VP, VP]),
        "lh_remap_apply": (I, [P, VP, VP, D, VP, VP, VP, VP]),
        "lh_stiffness_setup": (I, [P, VP, VP]),
        "lh_stiffness_mult": (I, [P, VP, VP, VP]),
        "lh_laplacian": (I, [P, VP, VP, D, I, VP, VP]),
        "lh_tmop_objective": (I, [P, ctypes.POINTER(LhTmopParams), VP, VP, VP, VP]),
        "lh_tmop_gradient": (I, [P, ctypes.POINTER(LhTmopParams), VP, VP, VP, VP]),
        "lh_tmop_hessian_mult": (I, [P, ctypes.POINTER(LhTmopParams), VP, VP, VP, VP]),
        "lh_tmop_hessian_diag": (I, [P, ctypes.POINTER(LhTmopParams), VP, VP, VP]),
        "lh_tmop_workspace_size": (I, [P, ctypes.POINTER(ctypes.c_int64)]),
        "lh_tmop_hessian_setup": (I, [P, ctypes.POINTER(LhTmopParams), VP, VP, VP]),
        "lh_tmop_hessian_mult_pa": (I, [P, ctypes.POINTER(LhTmopParams), VP, VP, VP, VP]),
        "lh_timing_read": (I, [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I)]),
        "lh_learn_stats": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                               ctypes.POINTER(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class LhError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def _ptr(t):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class Sizes:
    ne: int
    n_h1: int
    nv: int
    n_l2: int
    nq: int
    arena_bytes: int


def mass_mult_noalloc(dim, n, order, q1, mq, x, y):
    """y = M_v x through lh_mass_mult_noalloc (no context, no device allocation).

    For callers that may not allocate device memory: mq ([NE][q1^dim] quadrature
    data omega*rho0*detJ0), x and y are caller-owned CUDA tensors."""
    import torch
    lib = load_library()
    nx, ny, nz = (n, n, n if dim == 3 else 1) if np.isscalar(n) else (tuple(n) + (1,))[:3]
    if dim == 2:
        nz = 1
    ne = nx * ny * nz
    n_h1 = (nx * order + 1) * (ny * order + 1) * ((nz * order + 1) if dim == 3 else 1)
    # the C ABI takes bare pointers: every length is checked here, before the call
    for name, t, need in (("mq", mq, ne * q1 ** dim), ("x", x, dim * n_h1), ("y", y, dim * n_h1)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError(f"mass_mult_noalloc: {name} must be a contiguous float64 CUDA tensor")
        if t.numel() < need:
            raise ValueError(f"mass_mult_noalloc: {name} has {t.numel()} values, needs {need}")
    st = lib.lh_mass_mult_noalloc(dim, nx, ny, nz, order, q1, _ptr(mq), _ptr(x), _ptr(y), _stream())
    if st != LH_OK:
        raise LhError(st, lib.lh_last_error(None).decode())


class Context:
    """One problem instance: owns an lh_ctx (mesh, tables, quadrature data, arena)."""

    def __init__(self, dim: int, n, vertices: np.ndarray, order: int, q1: int, gamma: float = 5.0 / 3.0,
                 cfl: float = 0.5, use_viscosity: bool = True, source: str = "none", precision: str = "fp64",
                 rho0=None):
        import torch
        self.lib = load_library()
        nx, ny, nz = (n, n, n if dim == 3 else 1) if np.isscalar(n) else (tuple(n) + (1,))[:3]
        self.dim, self.order, self.q1 = dim, order, q1
        V = np.ascontiguousarray(vertices, dtype=np.float64)
        self._verts = V
        prm = LhParams(dim, nx, ny, nz, V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), order, q1,
                       float(gamma), float(cfl), int(bool(use_viscosity)), SOURCES[source], PRECISIONS[precision])
        h = ctypes.c_void_p()
        st = self.lib.lh_setup(ctypes.byref(prm), _ptr(rho0), ctypes.byref(h))
        if st != LH_OK:
            raise LhError(st, self.lib.lh_last_error(None).decode())
        self.h = h
        s = LhSizes()
        self._check(self.lib.lh_get_sizes(self.h, ctypes.byref(s)))
        self.sizes = Sizes(s.ne, s.n_h1, s.nv, s.n_l2, s.nq, s.arena_bytes)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def _check(self, st):
        if st != LH_OK:
            raise LhError(st, self.lib.lh_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.lh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- buffers -------------------------------------------------------------
    def h1_vector(self):
        import torch
        return torch.zeros((self.dim, self.sizes.n_h1), dtype=torch.float64, device=self.device)

    def l2_vector(self):
        import torch
        return torch.zeros((self.sizes.ne, self.sizes.n_l2 // self.sizes.ne), dtype=torch.float64,
                           device=self.device)

    def new_step_info(self, t: float = 0.0, t_end: float = 0.0):
        import torch
        info = LhStepInfo()
        info.t, info.t_end = t, t_end
        raw = np.frombuffer(bytes(info), dtype=np.uint8).copy()
        return torch.from_numpy(raw).to(self.device)

    @staticmethod
    def read_step_info(buf) -> LhStepInfo:
        return LhStepInfo.from_buffer_copy(buf.cpu().numpy().tobytes())

    def new_cg_info(self):
        import torch
        return torch.zeros(ctypes.sizeof(LhCgInfo), dtype=torch.uint8, device=self.device)

    @staticmethod
    def read_cg_info(buf) -> LhCgInfo:
        return LhCgInfo.from_buffer_copy(buf.cpu().numpy().tobytes())

    # --- C ABI calls (same names) --------------------------------------------
    def init_state(self, problem: str = "taylor_green"):
        x, v, e = self.h1_vector(), self.h1_vector(), self.l2_vector()
        self._check(self.lib.lh_init_state(self.h, PROBLEMS[problem], _ptr(x), _ptr(v), _ptr(e), _stream()))
        return x, v, e

    def update_qdata(self, x, v, e, dt_est=None):
        self._check(self.lib.lh_update_qdata(self.h, _ptr(x), _ptr(v), _ptr(e), _ptr(dt_est), _stream()))

    def copy_qdata(self, out):
        self._check(self.lib.lh_copy_qdata(self.h, _ptr(out), _stream()))

    def force_mult(self, u, rhs):
        self._check(self.lib.lh_force_mult(self.h, _ptr(u), _ptr(rhs), _stream()))

    def force_mult_t(self, v, out):
        self._check(self.lib.lh_force_mult_t(self.h, _ptr(v), _ptr(out), _stream()))

    def mass_mult(self, x, y):
        self._check(self.lib.lh_mass_mult(self.h, _ptr(x), _ptr(y), _stream()))

    def mass_mult_tc(self, x, y):
        """y = M x with the tensor-core element operator (FP32 tensors; bf16tc_ir contexts)."""
        self._check(self.lib.lh_mass_mult_tc(self.h, _ptr(x), _ptr(y), _stream()))

    def mass_cg(self, b, x, rel_tol=1e-12, max_it=1000, info=None):
        self._check(self.lib.lh_mass_cg(self.h, _ptr(b), _ptr(x), float(rel_tol), int(max_it), _ptr(info),
                                        _stream()))

    def energy_solve(self, rhs, out):
        self._check(self.lib.lh_energy_solve(self.h, _ptr(rhs), _ptr(out), _stream()))

    def rk2avg_step(self, x, v, e, dt, info, rel_tol=1e-12, max_it=1000):
        self._check(self.lib.lh_rk2avg_step(self.h, _ptr(x), _ptr(v), _ptr(e), float(dt), float(rel_tol),
                                            int(max_it), _ptr(info), _stream()))

    def new_remap_info(self):
        import torch
        return torch.zeros(ctypes.sizeof(LhRemapInfo), dtype=torch.uint8, device=self.device)

    @staticmethod
    def read_remap_info(buf) -> LhRemapInfo:
        return LhRemapInfo.from_buffer_copy(buf.cpu().numpy().tobytes())

    def remap_velocity(self, x0, x1, v, steps, constrained=True, rel_tol=1e-12, max_it=1000, info=None):
        self._check(self.lib.lh_remap_velocity(self.h, _ptr(x0), _ptr(x1), _ptr(v), int(steps),
                                               1 if constrained else 0, float(rel_tol), int(max_it), _ptr(info),
                                               _stream()))

    def remap_apply(self, x0, x1, tau, v, kv=None, mv=None):
        self._check(self.lib.lh_remap_apply(self.h, _ptr(x0), _ptr(x1), float(tau), _ptr(v), _ptr(kv), _ptr(mv),
                                            _stream()))

    def stiffness_setup(self, x):
        self._check(self.lib.lh_stiffness_setup(self.h, _ptr(x), _stream()))

    def stiffness_mult(self, u, y):
        self._check(self.lib.lh_stiffness_mult(self.h, _ptr(u), _ptr(y), _stream()))

    def laplacian(self, v, lap, rel_tol=1e-12, max_it=1000, info=None):
        self._check(self.lib.lh_laplacian(self.h, _ptr(v), _ptr(lap), float(rel_tol), int(max_it), _ptr(info),
                                          _stream()))

    @staticmethod
    def _tmop_prm(h, gamma, dlim):
        return ctypes.byref(LhTmopParams(float(h), float(gamma), float(dlim)))

    def tmop_objective(self, x, x0, out, h, gamma=0.0, dlim=1.0):
        """F(x) into the DEVICE float64 tensor `out` (one element)."""
        self._check(self.lib.lh_tmop_objective(self.h, self._tmop_prm(h, gamma, dlim), _ptr(x), _ptr(x0),
                                               _ptr(out), _stream()))

    def tmop_gradient(self, x, x0, g, h, gamma=0.0, dlim=1.0):
        self._check(self.lib.lh_tmop_gradient(self.h, self._tmop_prm(h, gamma, dlim), _ptr(x), _ptr(x0), _ptr(g),
                                              _stream()))

    def tmop_hessian_mult(self, x, u, y, h, gamma=0.0, dlim=1.0):
        self._check(self.lib.lh_tmop_hessian_mult(self.h, self._tmop_prm(h, gamma, dlim), _ptr(x), _ptr(u),
                                                  _ptr(y), _stream()))

    def tmop_hessian_diag(self, x, diag, h, gamma=0.0, dlim=1.0):
        self._check(self.lib.lh_tmop_hessian_diag(self.h, self._tmop_prm(h, gamma, dlim), _ptr(x), _ptr(diag),
                                                  _stream()))

    def tmop_workspace(self):
        """A DEVICE float64 workspace for the partially assembled TMOP Hessian."""
        import torch
        n = ctypes.c_int64(0)
        self._check(self.lib.lh_tmop_workspace_size(self.h, ctypes.byref(n)))
        return torch.empty(int(n.value), dtype=torch.float64, device=self.device)

    def tmop_hessian_setup(self, x, work, h, gamma=0.0, dlim=1.0):
        self._check(self.lib.lh_tmop_hessian_setup(self.h, self._tmop_prm(h, gamma, dlim), _ptr(x), _ptr(work),
                                                   _stream()))

    def tmop_hessian_mult_pa(self, work, u, y, h, gamma=0.0, dlim=1.0):
        self._check(self.lib.lh_tmop_hessian_mult_pa(self.h, self._tmop_prm(h, gamma, dlim), _ptr(work), _ptr(u),
                                                     _ptr(y), _stream()))

    def sync_status(self) -> int:
        return int(self.lib.lh_sync_status(self.h))

    def set_dt_control(self, enable: bool = True) -> None:
        """Step control with rejection for CFL steps (lh_set_dt_control)."""
        self._check(self.lib.lh_set_dt_control(self.h, 1 if enable else 0))

    def timing_enable(self, enable: bool = True) -> None:
        """Record CUDA events around every later mass-solver launch (lh_timing_enable)."""
        self._check(self.lib.lh_timing_enable(self.h, 1 if enable else 0))

    def timing_read(self):
        """(summed solver milliseconds, number of solves) since the previous read."""
        ms, n = ctypes.c_double(0.0), ctypes.c_int(0)
        self._check(self.lib.lh_timing_read(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value


class Batch:
    """Independent problems advanced together (lh_batch_*): one persistent launch
    per hot-path operation for all problems, the step replayed as a CUDA graph."""

    def __init__(self, contexts, states, dts):
        import torch
        self.lib = load_library()
        n = len(contexts)
        self.contexts = list(contexts)
        self.states = list(states)
        P = ctypes.c_void_p
        ctx_arr = (P * n)(*[c.h for c in contexts])
        xs = (P * n)(*[_ptr(s[0]) for s in states])
        vs = (P * n)(*[_ptr(s[1]) for s in states])
        es = (P * n)(*[_ptr(s[2]) for s in states])
        dt_arr = (ctypes.c_double * n)(*[float(d) for d in dts])
        raw = np.zeros(n * ctypes.sizeof(LhStepInfo), dtype=np.uint8)
        self.infos = torch.from_numpy(raw).to(contexts[0].device)
        h = ctypes.c_void_p()
        st = self.lib.lh_batch_create(n, ctx_arr, xs, vs, es, dt_arr, _ptr(self.infos), ctypes.byref(h))
        if st != LH_OK:
            raise LhError(st, self.lib.lh_last_error(None).decode())
        self.h = h
        self.n = n

    def _check(self, st):
        if st != LH_OK:
            raise LhError(st, self.lib.lh_batch_last_error(self.h).decode())

    @staticmethod
    def _cfg_dict(c):
        return {"tiles": list(c[0:4]), "tiles_cg": list(c[4:8]), "threads": int(c[8])}

    def autotune(self):
        """Pick the tile shapes by timing whole steps (the state is left unchanged)."""
        cfg = (ctypes.c_int * 9)()
        self._check(self.lib.lh_batch_autotune(self.h, cfg))
        return self._cfg_dict(cfg)

    def set_config(self, tiles=(1, 1, 1, 1), tiles_cg=(1, 1, 1, 1), threads=256):
        cfg = (ctypes.c_int * 9)(*(list(tiles) + list(tiles_cg) + [int(threads)]))
        self._check(self.lib.lh_batch_set_config(self.h, cfg))

    def step(self, rel_tol=1e-12, max_it=1000):
        self._check(self.lib.lh_batch_step(self.h, float(rel_tol), int(max_it), _stream()))

    def read_infos(self):
        raw = self.infos.cpu().numpy().tobytes()
        sz = ctypes.sizeof(LhStepInfo)
        return [LhStepInfo.from_buffer_copy(raw[i * sz:(i + 1) * sz]) for i in range(self.n)]

    def close(self):
        if getattr(self, "h", None):
            self.lib.lh_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_IN, MLP_IN_PAD, MLP_HID, MLP_OUT = 586, 592, 128, 192


class MLP:
    """The learned-form per-element MLP (lh_mlp_*); training and inference run in liblh's kernels."""

    def __init__(self, seed=0, max_rows=1 << 17):
        import torch
        self.lib = load_library()
        h = ctypes.c_void_p()
        st = self.lib.lh_mlp_create(int(seed), int(max_rows), ctypes.byref(h))
        if st != LH_OK:
            raise LhError(st, self.lib.lh_last_error(None).decode())
        self.h = h
        self.max_rows = max_rows
        self.nparams = self.lib.lh_mlp_num_params()
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")

    def _check(self, st):
        if st != LH_OK:
            raise LhError(st, self.lib.lh_mlp_last_error(self.h).decode())

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparams, dtype=np.float32)
        self._check(self.lib.lh_mlp_get_params(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == self.nparams
        self._check(self.lib.lh_mlp_set_params(self.h, w.ctypes.data_as(ctypes.c_void_p)))

    def forward(self, X, Y):
        self._check(self.lib.lh_mlp_forward(self.h, _ptr(X), int(X.shape[0]), _ptr(Y), _stream()))

    def gradients(self, X, T, grads=None):
        self._check(self.lib.lh_mlp_gradients(self.h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(grads),
                                              _ptr(self.loss), _stream()))
        return self.loss

    def sync_status(self) -> int:
        """LH_ERR_TIMEOUT if a GEMM of this MLP gave up a bounded wait (cleared), else 0."""
        return int(self.lib.lh_mlp_sync_status(self.h))

    def train_step(self, X, T, lr):
        self._check(self.lib.lh_mlp_train_step(self.h, _ptr(X), _ptr(T), int(X.shape[0]), float(lr),
                                               _ptr(self.loss), _stream()))
        return self.loss

    def close(self):
        if getattr(self, "h", None):
            self.lib.lh_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def learn_attach(ctx, mlp, mode, X_buf=None, T_buf=None):
    """Attach the learned form to a context: mode 1 records (X_buf, T_buf rows), 2 predicts, 0 detaches."""
    cap = 0 if X_buf is None else int(X_buf.shape[0])
    ctx._check(ctx.lib.lh_learn_attach(ctx.h, mlp.h if mlp is not None else None, int(mode), _ptr(X_buf),
                                       _ptr(T_buf), cap))


def learn_set_record_stride(ctx, stride):
    """Recording keeps every stride-th element of each solve (rotating subset)."""
    ctx._check(ctx.lib.lh_learn_set_record_stride(ctx.h, int(stride)))


def learn_stats(ctx):
    vals = [ctypes.c_int() for _ in range(4)]
    ratio = ctypes.c_double()
    ctx._check(ctx.lib.lh_learn_stats(ctx.h, *[ctypes.byref(v) for v in vals], ctypes.byref(ratio)))
    return dict(rows=vals[0].value, solves=vals[1].value, predictions=vals[2].value, used=vals[3].value,
                mean_residual_ratio=ratio.value)
