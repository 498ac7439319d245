"""ctypes declarations of libdd.so (include/dd.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdd.so")
# DD_DEBUG_LIB=1 in the environment (read at the first load) selects the debug build:
# the same library with bounds checks in the kernels that record DD_ERR_ARG in the
# plan's device status word
LIB_DEBUG_PATH = os.path.join(HERE, "_build", "libdd_debug.so")

c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_dbl = ctypes.c_double
c_vp = ctypes.c_void_p
c_f32 = ctypes.c_float

DD_U8, DD_F32 = 0, 1

STATUS = {
    0: "DD_OK", 1: "DD_ERR_ARG", 2: "DD_ERR_OVERFLOW", 3: "DD_ERR_OOM", 4: "DD_ERR_CUDA",
    5: "DD_ERR_STATE", 6: "DD_ERR_TIMEOUT", 7: "DD_ERR_CAPACITY", 8: "DD_ERR_UNSUPPORTED",
}


class DDError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


class dd_band(ctypes.Structure):
    _fields_ = [
        ("nchan", c_i32),
        ("f_lo_mhz", c_dbl),
        ("df_mhz", c_dbl),
        ("descending", c_i32),
        ("dt_ms", c_dbl),
        ("nsamp", c_i64),
        ("in_type", c_i32),
        ("k_dm", c_dbl),
    ]


class dd_candidate(ctypes.Structure):
    _fields_ = [("dm_index", c_i32), ("width_index", c_i32), ("t", c_i32), ("snr", c_f32)]


# name -> (restype, argtypes); every symbol that include/dd.h declares
SIGNATURES = {
    "dd_trial_dms": (c_i32, [ctypes.POINTER(dd_band), c_dbl, c_dbl, c_i32, c_dbl, c_i32, c_vp, c_vp]),
    "dd_plan_create": (c_i32, [ctypes.POINTER(c_vp), ctypes.POINTER(dd_band), c_vp, c_i32]),
    "dd_set_profiles": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i32]),
    "dd_set_weights_device": (c_i32, [c_vp, c_vp, c_i32, c_vp]),
    "dd_plan_info": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "dd_get_tables": (c_i32, [c_vp, c_vp, c_vp]),
    "dd_dedisperse": (c_i32, [c_vp, c_vp, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp]),
    "dd_channel_stats": (c_i32, [c_vp, c_vp, c_i64, c_i64, c_i64, c_vp, c_vp, c_vp]),
    "dd_boxcar_snr": (c_i32, [c_vp, c_vp, c_i64, c_i64, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp,
                              c_f32, c_vp, c_i32, c_vp, c_vp]),
    "dd_boxcar_snr_noalloc": (c_i32, [c_vp, c_vp, c_i64, c_i64, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp,
                                      c_f32, c_vp, c_i32, c_vp, c_vp]),
    "dd_dedisperse_boxcar": (c_i32, [c_vp, c_vp, c_i64, c_i64, c_i64, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp,
                                     c_f32, c_vp, c_i32, c_vp, c_vp]),
    "dd_test_set_fused_parts": (c_i32, [c_vp, c_i32]),
    "dd_backward": (c_i32, [c_vp, c_vp, c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_vp, c_i64, c_vp]),
    "dd_plan_set_schedule": (c_i32, [c_vp, c_i32, c_i32]),
    "dd_plan_get_schedule": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "dd_plan_set_method": (c_i32, [c_vp, c_i32]),
    "dd_alu_peak": (c_i32, [c_i32, c_vp, c_vp]),
    "dd_predict_rect": (c_i32, [c_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, c_i32, c_vp]),
    "dd_select_samples": (c_i32, [c_vp, c_i32, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "dd_exact_profiles": (c_i32, [c_vp, ctypes.c_double, c_vp, c_vp]),
    "dd_select_profiles": (c_i32, [c_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "dd_detector_profile": (c_i32, [c_vp, c_i32, c_i32, c_vp, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "dd_plan_get_method": (c_i32, [c_vp, c_vp]),
    "dd_plan_autotune": (c_i32, [c_vp, c_vp, c_i64, c_vp, c_i64, ctypes.c_char_p, c_vp, c_vp]),
    "dd_batch_create": (c_i32, [c_vp, c_vp, c_i32]),
    "dd_batch_bind": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "dd_batch_dedisperse": (c_i32, [c_vp, c_vp]),
    "dd_batch_bind_boxcar": (c_i32, [c_vp, c_vp, c_i32, c_vp, c_vp, c_vp, c_vp]),
    "dd_batch_run": (c_i32, [c_vp, c_vp]),
    "dd_batch_capture": (c_i32, [c_vp, c_vp]),
    "dd_batch_replay": (c_i32, [c_vp, c_vp]),
    "dd_batch_info": (c_i32, [c_vp, c_vp, c_vp, c_vp]),
    "dd_batch_destroy": (c_i32, [c_vp]),
    "dd_get_device_status": (c_i32, [c_vp, c_vp, c_vp]),
    "dd_test_set_wait": (c_i32, [c_vp, c_i32, c_i64]),
    "dd_plan_destroy": (c_i32, [c_vp]),
    "dd_status_str": (ctypes.c_char_p, [c_i32]),
    "dd_version": (c_i32, []),
}

_lib = None


def load():
    """Loads the in-tree libdd.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = LIB_DEBUG_PATH if os.environ.get("DD_DEBUG_LIB", "") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{os.path.basename(path)} is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int, what: str) -> None:
    if code != 0:
        raise DDError(code, what)
