"""ctypes binding of libodwf.so: the C-ABI entry points under their own names.

Argument marshalling only: field arguments are numpy arrays (host memory) or torch
tensors (device memory), passed as raw pointers; streams are torch streams or raw
cudaStream_t integers.  There is no fallback: if the library is missing or does not
load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ODWF_LIBRARY selects another build of the same C ABI (e.g. the bounds-checked libodwf_check.so)
LIB_PATH = os.environ.get("ODWF_LIBRARY") or os.path.join(_HERE, "libodwf.so")

ODWF_OK, ODWF_EINVAL, ODWF_ENOMEM, ODWF_ENOCONV, ODWF_EBREAKDOWN, ODWF_ETIMEOUT, ODWF_ECUDA, ODWF_PENDING, \
    ODWF_ENOTFOUND, ODWF_ECANCELED, ODWF_EBUSY = range(11)
ODWF_F64, ODWF_F32, ODWF_F16, ODWF_BF16, ODWF_FF = range(5)
ODWF_MODE_FULL, ODWF_MODE_SCHUR_EVEN = 0, 1
ODWF_SYS_SCHUR_NORMAL, ODWF_SYS_FULL_NORMAL, ODWF_SYS_FULL_DIRAC = 0, 1, 2
ODWF_OMEGA_SHIFTED_R5, ODWF_OMEGA_PLAIN = 0, 1
ODWF_UPDATES_AUTO, ODWF_UPDATES_F64, ODWF_UPDATES_FF = 0, 1, 2

STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOCONV", 4: "EBREAKDOWN", 5: "ETIMEOUT", 6: "ECUDA",
                7: "PENDING", 8: "ENOTFOUND", 9: "ECANCELED", 10: "EBUSY"}


class odwf_lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 4), ("t_antiperiodic", ctypes.c_int32)]


class odwf_solve_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("delta", ctypes.c_double), ("system", ctypes.c_int32), ("link_recon", ctypes.c_int32),
                ("mq", ctypes.c_double), ("check_every", ctypes.c_int32), ("link_prec", ctypes.c_int32),
                ("update_arith", ctypes.c_int32)]


class odwf_solve_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("n_reliable", ctypes.c_int32), ("true_resid", ctypes.c_double),
                ("time_ms", ctypes.c_double), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class odwf_request(ctypes.Structure):
    _fields_ = [("field_id", ctypes.c_int32), ("Ns", ctypes.c_int32), ("m0", ctypes.c_double),
                ("mq", ctypes.c_double), ("omega", ctypes.POINTER(ctypes.c_double)), ("nrhs", ctypes.c_int32),
                ("b", ctypes.POINTER(ctypes.c_void_p)), ("x", ctypes.POINTER(ctypes.c_void_p)),
                ("tol", ctypes.c_double), ("prec", ctypes.c_int32), ("max_iter", ctypes.c_int32)]


class odwf_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("true_resid", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]


class odwf_kernel_prof(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("system_launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("bytes_per_system", ctypes.c_double),
                ("bytes_per_launch", ctypes.c_double)]


class odwf_cg_step_scalars(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("rr", ctypes.c_double), ("pAp", ctypes.c_double),
                ("alpha", ctypes.c_double), ("rr_new", ctypes.c_double), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class odwf_flow_obs(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("e_plaq", ctypes.c_double), ("e_clover", ctypes.c_double),
                ("q_clover", ctypes.c_double), ("plaq_min", ctypes.c_double), ("plaq_mean", ctypes.c_double)]


class OdwfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(code, "?"), code, msg))
        self.code = code


_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double

_SIGS = {
    "odwf_last_error": ([], ctypes.c_char_p),
    "odwf_version": ([], ctypes.c_char_p),
    "odwf_zolotarev_omega": ([I, D, D, I, P, P], I),
    "odwf_create": ([ctypes.POINTER(odwf_lattice), I, D, D, P, ctypes.POINTER(P)], I),
    "odwf_destroy": ([P], I),
    "odwf_set_gauge": ([P, P, P], I),
    "odwf_apply": ([P, P, P, I, P], I),
    "odwf_apply_dagger": ([P, P, P, I, P], I),
    "odwf_apply_normal": ([P, P, P, I, P], I),
    "odwf_apply_normal_prec": ([P, P, P, I, I, P], I),
    "odwf_apply_m5": ([P, P, P, ctypes.c_long, I, P], I),
    "odwf_apply_m5_noalloc": ([I, D, D, P, P, P, ctypes.c_long, I, P], I),
    "odwf_mixed_cg_step": ([P, I, I, I, D, P, P, P, P, ctypes.POINTER(odwf_cg_step_scalars), P], I),
    "odwf_cg_solve": ([P, P, P, ctypes.POINTER(odwf_solve_params), P, P], I),
    "odwf_effective_solve": ([P, P, P, ctypes.POINTER(odwf_solve_params), P, P], I),
    "odwf_residual_mass": ([P, P, ctypes.POINTER(odwf_solve_params), ctypes.POINTER(D), P, P, P], I),
    "odwf_cg_solve_batched": ([P, I, P, P, P, ctypes.POINTER(odwf_solve_params), P, P], I),
    "odwf_profile_enable": ([I], I),
    "odwf_profile_read": ([P, I, ctypes.POINTER(ctypes.c_int)], I),
    "odwf_launch_count": ([], ctypes.c_longlong),
    "odwf_time_kernel": ([P, I, I, I, I, I, I, P, P, P], I),
    "serve_create": ([ctypes.c_size_t, ctypes.POINTER(P)], I),
    "serve_register_gauge": ([P, I, ctypes.POINTER(odwf_lattice), P], I),
    "serve_submit": ([P, ctypes.POINTER(odwf_request), ctypes.POINTER(ctypes.c_uint64)], I),
    "serve_poll": ([P, ctypes.c_uint64, I, ctypes.POINTER(odwf_result)], I),
    "serve_destroy": ([P], I),
    "serve_set_policy": ([P, D, I, I], I),
    "serve_cancel": ([P, ctypes.c_uint64], I),
    "odwf_pf_force": ([P, P, D, D, ctypes.POINTER(odwf_solve_params), ctypes.POINTER(D), P, P, P], I),
    "odwf_pf_heatbath": ([P, P, D, D, ctypes.POINTER(odwf_solve_params), P, ctypes.POINTER(odwf_solve_stats), P], I),
    "odwf_gauge_force": ([P, P, D, ctypes.POINTER(D), P, P], I),
    "odwf_md_trajectory": ([P, P, P, I, P, P, P, D, D, I, I, I, ctypes.POINTER(odwf_solve_params), P,
                            ctypes.POINTER(odwf_solve_stats), P], I),
    "odwf_flow_create": ([ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(P)], I),
    "odwf_flow_destroy": ([P], I),
    "odwf_flow_set_gauge": ([P, P, P], I),
    "odwf_flow_get_gauge": ([P, P, P], I),
    "odwf_flow_measure": ([P, D, ctypes.POINTER(odwf_flow_obs), P, P, P], I),
    "odwf_flow_run": ([P, D, I, I, D, ctypes.POINTER(odwf_flow_obs), I, ctypes.POINTER(I), P], I),
    "odwf_flow_t0": ([ctypes.POINTER(odwf_flow_obs), I, D, ctypes.POINTER(D)], I),
}


def load(build_if_missing: bool = False):
    """Load libodwf.so (optionally building it first); raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from .build import build

            build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libodwf.so is not built (run __graft_entry__.build() or "
                               "python -m paper_1811_08095_gb300.build); there is no fallback path")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def check(code):
    if code != ODWF_OK:
        msg = load().odwf_last_error()
        raise OdwfError(code, msg.decode() if msg else "")
    return code


def ptr(a):
    """Raw pointer of a numpy array (host) or torch tensor (device or host)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data_as(ctypes.c_void_p)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    raise TypeError("unsupported field argument %r" % type(a))


def stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)
