"""ctypes loader for the in-tree CUDA library _build/libq2x.so (argument
marshalling only).  There is no fallback: if the library is missing or cannot
be loaded, every call raises."""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_build", "libq2x.so")
_LOCK = threading.Lock()
_LIB = None

Q2X_OK = 0
STATUS_NAMES = {0: "Q2X_OK", 1: "Q2X_ERR_ARG", 2: "Q2X_ERR_RANGE", 3: "Q2X_ERR_CUDA", 4: "Q2X_ERR_OOM",
                5: "Q2X_ERR_DEVICE_INPUT", 6: "Q2X_ERR_TIMEOUT", 7: "Q2X_ERR_UNSUPPORTED"}

_c = ctypes
_p, _i, _i64, _u32p = _c.c_void_p, _c.c_int, _c.c_int64, _c.POINTER(_c.c_uint32)
_ELEM = [_p, _i64, _i64, _p, _p, _p, _i64, _p, _p, _p, _p, _p, _i]  # segments / tetra
_SIGNATURES = {
    "q2x_plan": [_c.POINTER(_p), _i, _i, _i, _p],
    "q2x_plan_destroy": [_p],
    "q2x_plan_set_stream": [_p, _p],
    "q2x_plan_set_kernel_timing": [_p, _i],
    "q2x_plan_kernel_timing": [_p, _c.POINTER(_c.c_double), _c.POINTER(_i64)],
    "q2x_sync": [_p],
    "q2x_device_errors": [_p, _u32p],
    "q2x_reserve": [_p, _i64, _i64],
    "q2x_segments": _ELEM,
    "q2x_tetra": _ELEM,
    "q2x_triangles": [_p, _i64, _i64, _p, _p, _i, _p, _i64, _p, _p, _p, _p, _p, _p, _i],
    "q2x_triangles_single": [_p, _i64, _i64, _p, _p, _i, _p, _i64, _p, _p, _p, _p, _p, _i],
    "q2x_triangles_double": [_p, _i64, _i64, _p, _p, _i, _p, _i64, _p, _p, _p, _p, _p, _i],
    "q2x_leaf_reduce": [_p, _i64, _i, _p, _i64, _p, _p, _i],
    "q2x_translate": [_p, _i, _i64, _p, _p, _i64, _p, _p, _p, _i],
    "q2x_translation_rows": [_p, _i, _i64, _p, _p],
    "q2x_translate_rt": [_p, _i, _i64, _p, _i64, _p, _p, _i64, _p, _p, _i],
    "q2x_evaluate": [_p, _i, _i64, _p, _p, _i64, _p, _p, _p, _p, _i],
    "q2x_evaluate_curl": [_p, _i, _i64, _p, _p, _i64, _p, _p, _p, _p, _i],
    "q2x_segments_vector": [_p, _i64, _i64, _p, _p, _p, _i64, _p, _p, _p, _p, _p, _i],
    "q2x_leaf_reduce_weighted": [_p, _i64, _i, _p, _i, _p, _i64, _i64, _p, _p, _i64, _i],
    "q2x_nearfield": [_p, _i, _i, _i64, _i64, _p, _p, _p, _i64, _p, _p, _p, _p, _i],
    "q2x_galerkin_triangles": [_p, _i64, _i64, _p, _p, _p, _i64, _p, _p, _p, _i, _p, _p],
    "q2x_triangles_single_vjp": [_p, _i64, _i64, _p, _p, _p, _i64, _p, _p, _p, _p, _p, _p, _p],
    "q2x_batch_build": [_p, _p, _i, _c.POINTER(_p)],
    "q2x_batch_run": [_p],
    "q2x_batch_destroy": [_p],
    "q2x_batch_info": [_p, _c.POINTER(_i64), _c.POINTER(_i64), _c.POINTER(_i)],
    "q2x_batch_tune": [_p, _p, _p, _i, _i, _c.POINTER(_i), _c.POINTER(_c.c_float)],
    "q2x_alu_peak_probe": [_i, _i64, _p, _p, _c.POINTER(_c.c_double)],
}


class BatchElements(_c.Structure):
    """q2x_batch_elements"""
    _fields_ = [("n_elem", _i64), ("n_vert", _i64), ("vxyz", _p), ("idx", _p), ("sigma", _p),
                ("leaf_off", _p), ("density", _i)]


class BatchDesc(_c.Structure):
    """q2x_batch_desc"""
    _fields_ = [("n_leaves", _i64), ("leaf_c", _p), ("leaf_rho", _p), ("leaf_p", _p),
                ("segments", BatchElements), ("triangles", BatchElements), ("tetra", BatchElements),
                ("coef", _p), ("accumulate", _i)]


class Q2XError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


def lib():
    """Load libq2x.so (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(SO_PATH):
                raise RuntimeError("the Q2X CUDA library is not built (%s missing); run "
                                   "`python -m paper_2107_10942_gb300.build`" % SO_PATH)
            L = ctypes.CDLL(SO_PATH)
            for name, args in _SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = _c.c_int
            L.q2x_last_error.argtypes = [_p]
            L.q2x_last_error.restype = _c.c_char_p
            L.q2x_workspace_bytes.argtypes = [_p]
            L.q2x_workspace_bytes.restype = _c.c_int64
            L.q2x_launch_count.argtypes = [_p]
            L.q2x_launch_count.restype = _c.c_int64
            _LIB = L
    return _LIB


def check(status: int, plan=None):
    if status != Q2X_OK:
        msg = lib().q2x_last_error(plan)
        raise Q2XError(status, msg.decode() if msg else "")
