"""CPU checks of the boundary: the C-ABI library loads and exports every symbol include/lh.h declares."""
import ctypes
import os
import re

from paper_2112_07075_b300 import lh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lh.h")).read()
    return sorted(set(re.findall(r"^\s*(?:lh_status|void|int|const char \*)\s*\*?\s*(lh_\w+)\s*\(", src, re.M)))


def test_header_declares_the_binding_names():
    assert _declared() == sorted(lh.EXPORTED)


def test_library_exports_every_declared_symbol():
    lib = lh.load_library()
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_sizes_match_the_header():
    assert ctypes.sizeof(lh.LhStepInfo) == 104
    assert ctypes.sizeof(lh.LhCgInfo) == 32
    assert ctypes.sizeof(lh.LhParams) == 64
    assert ctypes.sizeof(lh.LhRemapInfo) == 32
    assert ctypes.sizeof(lh.LhTmopParams) == 24


def test_setup_rejects_bad_arguments_without_a_gpu():
    lib = lh.load_library()
    h = ctypes.c_void_p()
    assert lib.lh_setup(None, None, ctypes.byref(h)) == lh.LH_ERR_ARG
    import numpy as np
    V = np.zeros((4, 2))
    prm = lh.LhParams(4, 1, 1, 1, V.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 2, 4, 5 / 3, 0.5, 1, 0, 0)
    assert lib.lh_setup(ctypes.byref(prm), None, ctypes.byref(h)) == lh.LH_ERR_ARG
    assert b"dim" in lib.lh_last_error(None)
    prm.dim, prm.order = 2, 7
    assert lib.lh_setup(ctypes.byref(prm), None, ctypes.byref(h)) == lh.LH_ERR_ARG
    prm.order, prm.source = 2, 1
    prm.dim = 3
    assert lib.lh_setup(ctypes.byref(prm), None, ctypes.byref(h)) == lh.LH_ERR_ARG


def test_widened_entry_points_reject_null_arguments_without_a_gpu():
    """The remap, stiffness, TMOP and step-control calls check their arguments on the
    host before anything is enqueued (no device is touched)."""
    lib = lh.load_library()
    E = lh.LH_ERR_ARG
    prm = lh.LhTmopParams(0.25, 0.0, 1.0)
    assert lib.lh_remap_velocity(None, None, None, None, 1, 1, 0.0, 0, None, None) == E
    assert lib.lh_remap_apply(None, None, None, 0.5, None, None, None, None) == E
    assert lib.lh_stiffness_setup(None, None, None) == E
    assert lib.lh_stiffness_mult(None, None, None, None) == E
    assert lib.lh_laplacian(None, None, None, 0.0, 0, None, None) == E
    assert lib.lh_tmop_objective(None, ctypes.byref(prm), None, None, None, None) == E
    assert lib.lh_tmop_gradient(None, ctypes.byref(prm), None, None, None, None) == E
    assert lib.lh_tmop_hessian_mult(None, ctypes.byref(prm), None, None, None, None) == E
    assert lib.lh_tmop_hessian_diag(None, ctypes.byref(prm), None, None, None) == E
    assert lib.lh_set_dt_control(None, 1) == E
