"""ctypes view of libgpp's C-ABI (include/gpp.h, include/gpp_diag.h).

Argument marshalling only: every step of the sum runs in the library's CUDA kernels. If
the library has not been built, loading fails loudly; there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgpp.so")

GPP_OK = 0
STATUS = {0: "GPP_OK", -1: "GPP_ERR_NULL_PTR", -2: "GPP_ERR_BAD_SIZE", -3: "GPP_ERR_BAD_INDEX",
          -4: "GPP_ERR_WORKSPACE", -5: "GPP_ERR_CUDA", -6: "GPP_ERR_UNSUPPORTED",
          -7: "GPP_ERR_TIMEOUT", -8: "GPP_ERR_BAD_OPTION"}
GPP_FP64, GPP_FP32_BULK = 0, 1
GPP_OCC_ALL, GPP_OCC_OCCUPIED = 0, 1
GPP_MAX_NW = 8
GPP_PHYS_CH_HALF, GPP_PHYS_SX_CUTOFF = 1, 2
PEAK_KINDS = {"dfma": 0, "ffma": 1, "dadd": 2, "dmul": 3, "drcp": 4, "drcp_rn": 5,
              "drcp_approx": 6, "fsel": 7, "fsetp": 8, "isel": 9, "f2f": 10}
PEAK_CHAINS = 8

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


class GppProblem(ctypes.Structure):
    _fields_ = [("number_bands", _i64), ("nvband", _i64), ("ncouls", _i64), ("ngpown", _i64),
                ("nw", _i64),
                ("aqsmtemp", _vp), ("aqsntemp", _vp), ("I_eps_array", _vp),
                ("wtilde_array", _vp), ("vcoul", _vp), ("inv_igp_index", _vp), ("indinv", _vp),
                ("wx_array", _vp),
                ("aqsntemp_c64", _vp), ("achtemp", _vp), ("asxtemp", _vp)]


class GppGrads(ctypes.Structure):
    _fields_ = [("wtilde_array", _vp), ("I_eps_array", _vp), ("aqsmtemp", _vp),
                ("aqsntemp", _vp)]


class GppOptions(ctypes.Structure):
    _fields_ = [("precision", _i32), ("occ_mode", _i32), ("block_threads", _i32),
                ("blocks_per_sm", _i32), ("debug_checks", _i32), ("ig_per_thread", _i32),
                ("physics", _i32), ("reserved", _i32), ("stage_events", ctypes.POINTER(_vp)),
                ("sexcut", ctypes.c_double)]


# (name, restype, argtypes) of every exported function, in header order.
SIGNATURES = [
    ("gpp_options_default", None, [ctypes.POINTER(GppOptions)]),
    ("gpp_sigma_workspace_size", ctypes.c_size_t,
     [ctypes.POINTER(GppProblem), ctypes.POINTER(GppOptions)]),
    ("gpp_sigma", ctypes.c_int,
     [ctypes.POINTER(GppProblem), ctypes.POINTER(GppOptions), _vp, ctypes.c_size_t, _vp]),
    ("gpp_sigma_noalloc", ctypes.c_int,
     [ctypes.POINTER(GppProblem), ctypes.POINTER(GppOptions), _vp]),
    ("gpp_sigma_host_workspace_size", ctypes.c_size_t,
     [ctypes.POINTER(GppProblem), ctypes.POINTER(GppOptions)]),
    ("gpp_sigma_host", ctypes.c_int,
     [ctypes.POINTER(GppProblem), ctypes.POINTER(GppOptions), _vp, ctypes.c_size_t, _vp]),
    ("gpp_sigma_backward_workspace_size", ctypes.c_size_t,
     [ctypes.POINTER(GppProblem), ctypes.POINTER(GppOptions)]),
    ("gpp_sigma_backward", ctypes.c_int,
     [ctypes.POINTER(GppProblem), ctypes.POINTER(GppOptions), _vp, _vp,
      ctypes.POINTER(GppGrads), _vp, ctypes.c_size_t, _vp]),
    ("gpp_batched_workspace_size", ctypes.c_size_t,
     [ctypes.POINTER(GppProblem), ctypes.c_int, ctypes.POINTER(GppOptions)]),
    ("gpp_batched_plan_create", ctypes.c_int,
     [ctypes.POINTER(_vp), ctypes.POINTER(GppProblem), ctypes.c_int, ctypes.POINTER(GppOptions),
      _vp, ctypes.c_size_t, ctypes.c_int, _vp]),
    ("gpp_batched_plan_run", ctypes.c_int, [_vp, _vp]),
    ("gpp_batched_plan_destroy", ctypes.c_int, [_vp]),
    ("gpp_sigma_batched", ctypes.c_int,
     [ctypes.POINTER(GppProblem), ctypes.c_int, ctypes.POINTER(GppOptions), _vp,
      ctypes.c_size_t, _vp]),
    ("gpp_convert_c64", ctypes.c_int, [_vp, _vp, _i64, _vp]),
    ("gpp_last_error", ctypes.c_char_p, []),
    ("gpp_version", ctypes.c_char_p, []),
    ("gpp_peak_launch", ctypes.c_int, [ctypes.c_int, _i64, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    ("gpp_diag_rcp", ctypes.c_int, [_vp, _vp, _i64, _vp]),
    ("gpp_diag_inject_cuda_failure", None, [ctypes.c_int]),
]

_lock = threading.Lock()
_lib = None


class GppError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """The loaded libgpp (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"libgpp.so is not built ({LIB_PATH} missing): run "
                "`python -c 'import __graft_entry__ as g; g.build()'` first")
        handle = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
        return handle


def check(rc: int):
    if rc != GPP_OK:
        raise GppError(rc, lib().gpp_last_error().decode())


def options(precision=GPP_FP64, occ_mode=GPP_OCC_ALL, block_threads=0, blocks_per_sm=0,
            debug_checks=False, stage_events=None, ig_per_thread=0, ch_half=False,
            sexcut=0.0) -> GppOptions:
    o = GppOptions()
    lib().gpp_options_default(ctypes.byref(o))
    o.precision = precision
    o.occ_mode = occ_mode
    o.block_threads = block_threads
    o.blocks_per_sm = blocks_per_sm
    o.debug_checks = 1 if debug_checks else 0
    o.ig_per_thread = ig_per_thread
    o.physics = (GPP_PHYS_CH_HALF if ch_half else 0) | (GPP_PHYS_SX_CUTOFF if sexcut else 0)
    o.sexcut = float(sexcut)
    if stage_events is not None:
        arr = (_vp * 4)(*[ctypes.c_void_p(h) for h in stage_events])
        o._events_keepalive = arr
        o.stage_events = ctypes.cast(arr, ctypes.POINTER(_vp))
    return o
