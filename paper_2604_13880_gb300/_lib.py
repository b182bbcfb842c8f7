"""ctypes binding of libinim.so (the C ABI declared in include/inim.h).

Argument marshalling only: every step of the cartogram iteration runs in the
library's CUDA kernels.  Loading fails loudly when the library is missing; there
is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libinim.so")

INIM_OK = 0
INIM_E_ARG, INIM_E_VALUE, INIM_E_CUDA, INIM_E_TIMEOUT, INIM_E_CAPACITY, INIM_E_STATE = -1, -2, -3, -4, -5, -6
INIM_W_NOT_CONVERGED, INIM_W_FOLDOVER = 1, 2
INIM_DIRECT, INIM_CUMULATIVE = 0, 1
INIM_FP32, INIM_FIX64, INIM_KAHAN = 0, 1, 2
INIM_FORM_FUSED, INIM_FORM_PLAIN = 0, 1
INIM_MAP_DEVICE_PTRS = 1


class inim_params(ctypes.Structure):
    _fields_ = [
        ("log2_res", ctypes.c_int32),
        ("shape", ctypes.c_float),
        ("bdv_scale", ctypes.c_float),
        ("max_iters", ctypes.c_int32),
        ("xi_stop", ctypes.c_float),
        ("stall_window", ctypes.c_int32),
        ("eps_stop", ctypes.c_float),
        ("mode", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("form", ctypes.c_int32),
        ("warm_start", ctypes.c_int32),
        ("bdv_value", ctypes.c_float),
    ]


class inim_quality_out(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double),
        ("shape", ctypes.c_double),
        ("rel_pos", ctypes.c_double),
        ("adj_map", ctypes.c_int64),
        ("adj_cart", ctypes.c_int64),
        ("adj_both", ctypes.c_int64),
        ("n_present", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


class inim_step_stats(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int32),
        ("eps", ctypes.c_float),
        ("xi", ctypes.c_float),
        ("foldover", ctypes.c_int32),
        ("overlap", ctypes.c_int32),
        ("status", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class inim_job(ctypes.Structure):
    _fields_ = [
        ("map", ctypes.c_void_p),
        ("values", ctypes.c_void_p),
        ("init_xy", ctypes.c_void_p),
        ("out_xy", ctypes.c_void_p),
        ("params", inim_params),
        ("stats", ctypes.POINTER(inim_step_stats)),
    ]


class inim_series(ctypes.Structure):
    _fields_ = [
        ("map", ctypes.c_void_p),
        ("values", ctypes.c_void_p),
        ("T", ctypes.c_int32),
        ("init_xy", ctypes.c_void_p),
        ("out_xy", ctypes.c_void_p),
        ("params", inim_params),
        ("stats", ctypes.POINTER(inim_step_stats)),
    ]


# name -> (restype, argtypes)
_SIGS = {
    "inim_params_default": (None, [ctypes.POINTER(inim_params)]),
    "inim_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "inim_last_error": (ctypes.c_char_p, []),
    "inim_interpolate_values": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_void_p]),
    "inim_background_values": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_void_p, ctypes.c_void_p]),
    "inim_map_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_void_p)]),
    "inim_map_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "inim_map_info": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int32)] * 4),
    "inim_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(inim_params),
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(inim_step_stats),
                                ctypes.c_void_p]),
    "inim_run_batch": (ctypes.c_int, [ctypes.POINTER(inim_job), ctypes.c_int32, ctypes.c_void_p]),
    "inim_run_dynamic": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(inim_params),
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(inim_step_stats),
                                        ctypes.c_void_p]),
    "inim_run_series": (ctypes.c_int, [ctypes.POINTER(inim_series), ctypes.c_int32, ctypes.c_void_p]),
    "inim_set_persistent": (ctypes.c_int, [ctypes.c_int32]),
    "inim_persistent_phase_times": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.c_int32]),
    "inim_raster": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "inim_inims": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "inim_displacement": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                         ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "inim_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(inim_params),
                                    ctypes.c_int32, ctypes.POINTER(inim_step_stats), ctypes.c_void_p]),
    "inim_areas": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "inim_quality": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                    ctypes.POINTER(inim_quality_out), ctypes.c_void_p, ctypes.c_void_p]),
    "inim_inims_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "inim_density_pooled": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "inim_cnn_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "inim_cnn_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "inim_cnn_num_params": (ctypes.c_longlong, [ctypes.c_void_p]),
    "inim_cnn_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong]),
    "inim_cnn_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong]),
    "inim_cnn_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "inim_cnn_gradients": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_float), ctypes.c_void_p, ctypes.c_void_p]),
    "inim_cnn_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_float, ctypes.POINTER(ctypes.c_float), ctypes.c_void_p]),
    "inim_cnn_last_error": (ctypes.c_char_p, []),
    "inim_cnn_loss_mean": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "inim_warmstart_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t]),
    "inim_warmstart_load_res": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32]),
    "inim_cnn_create_res": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "inim_cnn_input_res": (ctypes.c_int, [ctypes.c_void_p]),
    "inim_set_scan_tile": (ctypes.c_int, [ctypes.c_int32] * 6),
    "inim_get_scan_tile": (ctypes.c_int, [ctypes.c_int32] * 3 + [ctypes.POINTER(ctypes.c_int32)] * 3),
    "inim_autotune_scan": (ctypes.c_int, [ctypes.POINTER(inim_job), ctypes.c_int32, ctypes.c_int32]),
    "inim_profile_stages": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_int32)]),
    "inim_stage_name": (ctypes.c_char_p, [ctypes.c_int32]),
    "inim_launch_count": (ctypes.c_longlong, []),
    "inim_set_wait_cap": (ctypes.c_int, [ctypes.c_int64]),
    "inim_set_single_pass_scan": (ctypes.c_int, [ctypes.c_int32]),
    "inim_set_area_overlap": (ctypes.c_int, [ctypes.c_int32]),
    "inim_timeline": (ctypes.c_int, [ctypes.c_int32]),
    "inim_timeline_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                          ctypes.c_int32]),
}

_lib = None


def load():
    """Load libinim.so once; raise if it is missing (no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libinim.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols():
    """Names of the functions the header declares (and the binding wraps)."""
    return list(_SIGS)


class InimError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.inim_last_error().decode()
        text = lib.inim_status_string(status).decode()
        super().__init__(f"{where}: {text} ({status}) {msg}")
        self.status = status


def check(status, where):
    if status < 0:
        raise InimError(status, where)
    return status


# ---------------------------------------------------------------------------
# pointer helpers (numpy host arrays or torch tensors)
# ---------------------------------------------------------------------------
def ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensors must be contiguous"
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def stream_of(*arrays):
    for a in arrays:
        if hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None



class CnnError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        super().__init__(f"{where}: {lib.inim_status_string(status).decode()} ({status}) "
                         f"{lib.inim_cnn_last_error().decode()}")
        self.status = status


def check_cnn(status, where):
    """Status check for the inim_cnn_* entry points (they keep their own error text)."""
    if status < 0:
        raise CnnError(status, where)
    return status
