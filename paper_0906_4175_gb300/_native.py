"""ctypes loader for libmfgb.so (the C ABI declared in include/mfgb.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# MFGB_DEBUG_LIB=1 loads the debug build (index checks, build.py --debug) instead
LIB_PATH = os.path.join(_PKG, "_build_debug" if os.environ.get("MFGB_DEBUG_LIB") == "1" else "_build", "libmfgb.so")

MF_OK, MF_EINVAL, MF_ENOMEM, MF_ECUDA, MF_EOVERFLOW, MF_ETIMEOUT, MF_ENOTSUP = range(7)
MF_PHASE_ANCHOR, MF_PHASE_FP64, MF_PHASE_FP32 = 0, 1, 2
MF_FFT_FP32, MF_FFT_TC_FP16, MF_FFT_TC_BF16 = 0, 1, 2
MF_COND_FP64, MF_COND_FP32 = 0, 1
_NAMES = {0: "MF_OK", 1: "MF_EINVAL", 2: "MF_ENOMEM", 3: "MF_ECUDA", 4: "MF_EOVERFLOW",
          5: "MF_ETIMEOUT", 6: "MF_ENOTSUP"}

# exported entry points (name -> (restype, argtypes)); include/mfgb.h is the reference
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_F = ctypes.c_float
SIGNATURES = {
    "mf_last_error": (ctypes.c_char_p, []),
    "mf_version": (ctypes.c_char_p, []),
    "mf_bank_create": (_I, [_P, _P, _I64, _P, _P]),
    "mf_bank_destroy": (_I, [_P]),
    "mf_bank_size": (_I, [_P, _P]),
    "mf_bank_partition": (_I, [_P, _P, _I64, _P, _P, _P, _I, _I, _P]),
    "mf_bank_create_shard": (_I, [_P, _P, _I64, _P, _I64, _I64, _P]),
    "mf_segment_upload": (_I, [_P, _I64, _D, _P, _D, _D, _I, _P, _P]),
    "mf_segment_destroy": (_I, [_P]),
    "mf_segment_refresh": (_I, [_P, _P, _I, _P]),
    "mf_segment_set_conditioning": (_I, [_P, _I]),
    "mf_segment_info": (_I, [_P, _P, _P]),
    "mf_filter_bank": (_I, [_P, _P, _I, _F, _P, _P, _I64, _P, _P]),
    "mf_bank_check": (_I, [_P, _P]),
    "mf_synth_segment": (_I, [_P, _I64, _D, _D, _P, _D, _D, _P, _I64, _D, _P, _P]),
    "mf_refine_triggers": (_I, [_P, _P, _P, _I64, _P, _P, _P, _P]),
    "mf_fft_c2c": (_I, [_P, _P, _I64, _I64, _I, _P]),
    "mf_cluster_triggers": (_I, [_P, _P, _I64, _I64, _I, _I64, ctypes.c_int32, _P, _I64, _P, _P]),
    "mf_chisq_points": (_I, [_P, _P, _I, _P, _I64, _I64, _I, _P, _P]),
    "mf_chisq_series": (_I, [_P, _P, _P, _I64, _I, _P, _P, _P]),
    "mf_refine_triggers_multi": (_I, [_P, _I, _P, _P, _P, _I64, _P, _P, _P, _P]),
    "mf_refine_triggers_static": (_I, [_P, _P, _P, _I64, _P, _P, _P, _P]),
    "mf_launch_count": (_I, [_P]),
    "mf_debug_status": (_I, [_P, _P]),
    "mf_bank_profile": (_I, [_P, _I]),
    "mf_bank_profile_read": (_I, [_P, _P, _P, _P]),
    "mf_bank_debug_stall": (_I, [_P, _I64, _I64]),
    "mf_debug_fail_alloc": (_I, [_I64]),
    "mf_autotune": (_I, [_P, _P, _I, _F, _I, ctypes.c_char_p, _P]),
}
STAGES = ("setup", "anchors", "pass1", "pass2", "final", "fused")


class BankParams(ctypes.Structure):
    _fields_ = [("f_low", ctypes.c_double), ("pn_order", ctypes.c_int), ("amp_order", ctypes.c_int),
                ("phase_mode", ctypes.c_int), ("fft_mode", ctypes.c_int)]


PEAK_DTYPE = np.dtype([("rho", "f4"), ("j", "i4"), ("z_re", "f4"), ("z_im", "f4")])
TRIG_DTYPE = np.dtype([("tmpl", "i4"), ("seg", "i4"), ("j", "i4"), ("rho", "f4"), ("z_re", "f4"),
                       ("z_im", "f4")])
EVENT_DTYPE = np.dtype([("tmpl", "i4"), ("seg", "i4"), ("j", "i4"), ("rho", "f4"), ("z_re", "f4"),
                        ("z_im", "f4"), ("n_trig", "i4"), ("n_tmpl", "i4")])
INJ_DTYPE = np.dtype([("m1", "f8"), ("m2", "f8"), ("snr", "f8"), ("j0", "i8"), ("phi", "f8")])


class MFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (_NAMES.get(code, str(code)), msg))
        self.code = code


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("libmfgb.so is not built (run paper_0906_4175_gb300.build.build()); "
                                  "there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(rc: int, allow=()):
    if rc != MF_OK and rc not in allow:
        raise MFError(rc, lib().mf_last_error().decode("utf-8", "replace"))
    return rc
