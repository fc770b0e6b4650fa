"""ctypes binding of ``libpppm.so`` (the C ABI declared in include/pppm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  If the library is missing the import of the functions fails loudly;
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpppm.so")

PPPM_OK = 0
PPPM_ERR_INVALID_ARG = -1
PPPM_ERR_BAD_MESH = -2
PPPM_ERR_BAD_ORDER = -3
PPPM_ERR_BAD_BOX = -4
PPPM_ERR_CUDA = -5
PPPM_ERR_TIMEOUT = -6
PPPM_ERR_NONFINITE = -7
PPPM_ERR_TOO_LARGE = -8
PPPM_FP32 = 1
PPPM_FP64 = 2
PPPM_CORR_CELL = 0
PPPM_CORR_STATED = 1
PPPM_FORWARD_TCGEN05 = 0
PPPM_FORWARD_MMA_SYNC = 1
PPPM_BATCH_PERSISTENT = 0
PPPM_BATCH_STAGED = 1
PPPM_BATCH_AUTO = 2


class PPPMError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = strerror(code) if _lib is not None else str(code)
        if code == PPPM_ERR_CUDA and _lib is not None:
            msg += ": " + _lib.pppm_last_error().decode()
        super().__init__(f"{what}: {msg} (code {code})" if what else f"{msg} (code {code})")


class Options(ctypes.Structure):
    _fields_ = [("prefactor", ctypes.c_double), ("alias", ctypes.c_int), ("tile", ctypes.c_int)]


_lib = None
_lock = threading.Lock()

vp = ctypes.c_void_p
i64 = ctypes.c_int64
dbl = ctypes.c_double
cint = ctypes.c_int

# name -> (restype, argtypes)
SIGNATURES = {
    "pppm_default_options": (cint, [ctypes.POINTER(Options)]),
    "pppm_create": (cint, [ctypes.POINTER(dbl), ctypes.POINTER(cint), cint, dbl, cint, ctypes.POINTER(vp)]),
    "pppm_set_options": (cint, [vp, ctypes.POINTER(Options)]),
    "pppm_get_options": (cint, [vp, ctypes.POINTER(Options)]),
    "pppm_reserve": (cint, [vp, i64]),
    "pppm_destroy": (None, [vp]),
    "pppm_strerror": (ctypes.c_char_p, [cint]),
    "pppm_last_error": (ctypes.c_char_p, []),
    "pppm_status": (cint, [vp]),
    "pppm_compute": (cint, [vp, vp, vp, vp, i64, vp, vp, vp]),
    "pppm_compute_f32": (cint, [vp, vp, vp, vp, i64, vp, vp, vp]),
    "pppm_compute_host": (cint, [vp, vp, vp, i64, vp, vp, vp]),
    "pppm_compute_host_f32": (cint, [vp, vp, vp, i64, vp, vp, vp]),
    "pppm_spread": (cint, [vp, vp, vp, vp, i64, vp]),
    "pppm_fft_r2c": (cint, [vp, vp, vp, vp]),
    "pppm_fft_c2r": (cint, [vp, vp, vp, vp]),
    "pppm_influence": (cint, [vp, vp]),
    "pppm_fields": (cint, [vp, vp, vp, vp, i64, vp]),
    "pppm_spread_noalloc": (cint, [ctypes.POINTER(dbl), ctypes.POINTER(cint), cint, vp, vp, vp, i64, vp]),
    "pppm_batch_create": (cint, [cint, ctypes.POINTER(dbl), ctypes.POINTER(cint), cint, dbl, ctypes.POINTER(vp)]),
    "pppm_batch_set": (cint, [vp, dbl, cint, ctypes.c_longlong]),
    "pppm_batch_set_dft": (cint, [vp, cint]),
    "pppm_batch_set_quantized": (cint, [vp, cint, dbl]),
    "pppm_batch_meshes": (cint, [vp, ctypes.POINTER(cint)]),
    "pppm_batch_tile": (cint, [vp]),
    "pppm_compute_batched": (cint, [vp, vp, vp, vp, vp, vp, vp, vp]),
    "pppm_batch_status": (cint, [vp]),
    "pppm_batch_destroy": (None, [vp]),
    "pppm_set_potential": (cint, [vp, cint]),
    "pppm_set_dependent_launch": (cint, [vp, cint]),
    "pppm_set_wait_limit": (cint, [vp, ctypes.c_longlong]),
    "pppm_batch_set_wait_probe": (cint, [vp, cint]),
    "pppm_batch_set_launch": (cint, [vp, cint]),
    "pppm_batch_launch": (cint, [vp]),
    "pppm_corr_create": (cint, [vp, ctypes.POINTER(vp)]),
    "pppm_corr_nparams": (cint, []),
    "pppm_corr_create_features": (cint, [vp, cint, ctypes.POINTER(vp)]),
    "pppm_corr_param_count": (cint, [vp]),
    "pppm_corr_feature_width": (cint, [vp]),
    "pppm_corr_set_weights": (cint, [vp, vp, dbl, dbl]),
    "pppm_corr_get_weights": (cint, [vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
    "pppm_corr_features": (cint, [vp, vp, vp, vp, vp, i64, vp, vp]),
    "pppm_corr_calibrate": (cint, [vp, vp, vp, vp, vp, i64, vp]),
    "pppm_corr_get_scales": (cint, [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
    "pppm_corr_targets": (cint, [vp, vp, vp, vp, vp, i64, vp]),
    "pppm_corr_set_forward": (cint, [vp, cint]),
    "pppm_corr_set_wait_limit": (cint, [vp, ctypes.c_longlong]),
    "pppm_corr_forward": (cint, [vp, vp, vp, i64, vp]),
    "pppm_corr_apply": (cint, [vp, vp, vp, vp, vp, i64, vp, vp, vp]),
    "pppm_corr_grad": (cint, [vp, vp, vp, vp, i64, vp, i64, vp, vp]),
    "pppm_corr_train_step": (cint, [vp, vp, vp, vp, i64, vp, i64, ctypes.c_float, vp]),
    "pppm_corr_save": (cint, [vp, ctypes.c_char_p]),
    "pppm_corr_load": (cint, [vp, ctypes.c_char_p]),
    "pppm_corr_destroy": (None, [vp]),
    "pppm_wc_fold": (cint, [vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp]),
    "pppm_wc_fold_f32": (cint, [vp, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp]),
    "pppm_graph_create": (cint, [vp, vp, vp, vp, i64, vp, vp, vp, ctypes.POINTER(vp)]),
    "pppm_graph_create_f32": (cint, [vp, vp, vp, vp, i64, vp, vp, vp, ctypes.POINTER(vp)]),
    "pppm_graph_launch": (cint, [vp, vp, vp, vp]),
    "pppm_graph_launch_f32": (cint, [vp, vp, vp, vp]),
    "pppm_graph_destroy": (None, [vp]),
    "pppm_profile_enable": (cint, [vp, cint]),
    "pppm_profile_read": (cint, [vp, vp, vp, cint]),
    "pppm_profile_name": (ctypes.c_char_p, [cint]),
}


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} not found: build it with paper_2504_15508_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().pppm_strerror(int(code)).decode()


def check(code: int, what: str = "") -> None:
    if code != PPPM_OK:
        raise PPPMError(code, what)
