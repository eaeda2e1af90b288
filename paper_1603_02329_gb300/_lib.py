"""ctypes declarations of the C ABI in ``include/pat.h`` (argument marshalling only).

The shared library ``libpat_gb300.so`` must have been built (``build.build()``); importing
this module raises if it is missing, so nothing silently falls back to another code path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

PAT_OK, PAT_EINVAL, PAT_ECUDA, PAT_ENOMEM, PAT_ENONFINITE, PAT_ETIMEOUT, PAT_EUNSUPPORTED = range(7)
PAT_F32, PAT_F64 = 0, 1
STATUS_NAMES = {0: "PAT_OK", 1: "PAT_EINVAL", 2: "PAT_ECUDA", 3: "PAT_ENOMEM", 4: "PAT_ENONFINITE",
                5: "PAT_ETIMEOUT", 6: "PAT_EUNSUPPORTED"}


class pat_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("pml", ctypes.c_int * 3), ("pml_alpha", ctypes.c_double)]


class pat_sensors(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("pos", ctypes.POINTER(ctypes.c_double)),
                ("index", ctypes.POINTER(ctypes.c_int64))]


class pat_plan_info_t(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("N", ctypes.c_int64), ("Ns", ctypes.c_int),
                ("Nt", ctypes.c_int), ("lossy", ctypes.c_int), ("precision", ctypes.c_int),
                ("dt", ctypes.c_double), ("c_ref", ctypes.c_double), ("path", ctypes.c_int),
                ("layout", ctypes.c_int * 2), ("tuned", ctypes.c_int), ("schedule", ctypes.c_int),
                ("spec_chunks", ctypes.c_int), ("tma", ctypes.c_int),
                ("zreg", ctypes.c_int), ("ywide", ctypes.c_int), ("zwide", ctypes.c_int), ("rowu1", ctypes.c_int)]


class pat_fista_opts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("lambda_", ctypes.c_double), ("step_scale", ctypes.c_double),
                ("kappa", ctypes.c_double), ("vartheta", ctypes.c_double), ("q_d", ctypes.c_int), ("q_c", ctypes.c_int),
                ("eps_d", ctypes.c_double), ("eps_c", ctypes.c_double), ("tv_rho", ctypes.c_double),
                ("n_tv", ctypes.c_int), ("max_iter", ctypes.c_int), ("recursion", ctypes.c_int),
                ("L", ctypes.c_double), ("L_coarse", ctypes.c_double), ("target_re", ctypes.c_double),
                ("p_exact", ctypes.c_void_p), ("coarse_weight", ctypes.c_double)]


class pat_fista_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("recursive_iters", ctypes.c_int), ("fwd_solves", ctypes.c_int),
                ("adj_solves", ctypes.c_int), ("F", ctypes.c_double), ("RES", ctypes.c_double), ("RE", ctypes.c_double)]


ITER_CB = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                           ctypes.c_double, ctypes.c_int, ctypes.c_int)


class PatError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run paper_1603_02329_gb300.build.build() (needs nvcc)")
    L = ctypes.CDLL(path)
    vp, i32, f64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
    plan_pp = ctypes.POINTER(ctypes.c_void_p)
    L.pat_plan_create.argtypes = [ctypes.POINTER(pat_grid), dp, dp, dp, i32, f64, ctypes.POINTER(pat_sensors), f64, i32,
                                  i32, plan_pp]
    L.pat_plan_create.restype = i32
    L.pat_plan_destroy.argtypes = [vp]
    L.pat_plan_destroy.restype = i32
    L.pat_plan_get_info.argtypes = [vp, ctypes.POINTER(pat_plan_info_t)]
    L.pat_plan_get_info.restype = i32
    L.pat_forward_plan.argtypes = [vp, vp, vp, vp]
    L.pat_forward_plan.restype = i32
    L.pat_adjoint.argtypes = [vp, vp, vp, vp]
    L.pat_adjoint.restype = i32
    L.pat_plan_set_fault.argtypes = [vp, i32, f64]
    L.pat_plan_set_fault.restype = i32
    L.pat_plan_set_smoothing.argtypes = [vp, i32]
    L.pat_plan_set_smoothing.restype = i32
    L.pat_plan_smooth.argtypes = [vp, vp, vp, vp]
    L.pat_plan_smooth.restype = i32
    L.pat_gradient_c2.argtypes = [vp, vp, vp, vp, vp, i32, vp]
    L.pat_gradient_c2.restype = i32
    L.pat_gradient_rho.argtypes = [vp, vp, vp, vp, vp, i32, vp]
    L.pat_gradient_rho.restype = i32
    L.pat_gradient_medium.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp]
    L.pat_gradient_medium.restype = i32
    L.pat_probe_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), vp]
    L.pat_probe_fp32_peak.restype = i32
    L.pat_time_reversal.argtypes = [vp, vp, vp, i32, ctypes.c_double, vp]
    L.pat_time_reversal.restype = i32
    L.pat_adjoint_atd.argtypes = [vp, vp, vp, i32, vp]
    L.pat_adjoint_atd.restype = i32
    L.pat_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]
    L.pat_batch_create.restype = i32
    L.pat_batch_destroy.argtypes = [vp]
    L.pat_batch_destroy.restype = i32
    L.pat_batch_forward.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    L.pat_batch_forward.restype = i32
    L.pat_batch_adjoint.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    L.pat_batch_adjoint.restype = i32
    L.pat_forward.argtypes = [vp, dp, dp, dp, i32, f64, ctypes.POINTER(pat_grid), ctypes.POINTER(pat_sensors), f64, i32,
                              i32, vp, vp]
    L.pat_forward.restype = i32
    L.pat_forward_static.argtypes = L.pat_forward.argtypes
    L.pat_forward_static.restype = i32
    L.pat_plan_set_trace.argtypes = [vp, i32, i32]
    L.pat_plan_set_trace.restype = i32
    L.pat_plan_read_trace.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.c_size_t, ctypes.POINTER(i32)]
    L.pat_plan_read_trace.restype = i32
    L.pat_plan_status.argtypes = [vp]
    L.pat_plan_status.restype = i32
    L.pat_plan_set_probe.argtypes = [vp, i32]
    L.pat_plan_set_probe.restype = i32
    L.pat_plan_probe_slots.argtypes = [vp, i32]
    L.pat_plan_probe_slots.restype = i32
    L.pat_plan_probe_read.argtypes = [vp, i32, i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(f64),
                                      ctypes.POINTER(i32)]
    L.pat_plan_probe_read.restype = i32
    G = ctypes.POINTER(pat_grid)
    L.pat_tv_prox.argtypes = [G, vp, vp, f64, i32, i32, i32, vp]
    L.pat_tv_prox.restype = i32
    L.pat_tv.argtypes = [G, vp, f64, dp, i32, vp]
    L.pat_tv.restype = i32
    L.pat_tv_smooth_grad.argtypes = [G, vp, f64, vp, i32, vp]
    L.pat_tv_smooth_grad.restype = i32
    L.pat_restrict.argtypes = [G, vp, vp, i32, vp]
    L.pat_restrict.restype = i32
    L.pat_prolong.argtypes = [G, vp, vp, i32, vp]
    L.pat_prolong.restype = i32
    L.pat_coarse_bound.argtypes = [G, vp, vp, i32, vp]
    L.pat_coarse_bound.restype = i32
    L.pat_dot.argtypes = [vp, vp, ctypes.c_int64, i32, dp, vp]
    L.pat_dot.restype = i32
    L.pat_power_iteration.argtypes = [vp, vp, i32, dp, vp]
    L.pat_power_iteration.restype = i32
    L.pat_plan_create_coarse.argtypes = [vp, plan_pp]
    L.pat_plan_create_coarse.restype = i32
    L.pat_mg_fista.argtypes = [vp, vp, vp, vp, ctypes.POINTER(pat_fista_opts), vp, ctypes.POINTER(pat_fista_report),
                               ITER_CB, vp, vp]
    L.pat_mg_fista.restype = i32
    L.pat_mg_fista_levels.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(ctypes.c_double), vp, vp,
                                      ctypes.POINTER(pat_fista_opts), vp, ctypes.POINTER(pat_fista_report), ITER_CB,
                                      vp, vp]
    L.pat_mg_fista_levels.restype = i32
    L.pat_last_error.argtypes = []
    L.pat_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def check(status: int):
    if status != PAT_OK:
        msg = lib().pat_last_error().decode(errors="replace")
        raise PatError(status, msg)
