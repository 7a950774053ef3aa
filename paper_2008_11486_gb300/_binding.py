"""ctypes binding of the C ABI in include/irp.h (argument marshalling only).

Every function here forwards to the CUDA library ``_lib/libirp.so``; none
computes any step of the reduction.  If the library is missing the import of
the first call raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libirp.so")

IRP_OK = 0
STATUS_NAMES = {0: "IRP_OK", 1: "IRP_ERR_INVALID_ARG", 2: "IRP_ERR_ALIGNMENT",
                3: "IRP_ERR_WORKSPACE", 4: "IRP_ERR_UNSUPPORTED", 5: "IRP_ERR_BAD_MASTER",
                6: "IRP_ERR_CUDA", 7: "IRP_ERR_TIMEOUT", 8: "IRP_ERR_BAD_STATISTIC"}
INTERP = {"nearest": 0, "bilinear": 1, "spline3": 2, "cubic": 3}
FRAME_NORM = {"none": 0, "zero": 1, "scale": 2}
DTYPE = {"f32": 0, "f16": 1}
MAX_FRAMES = 64
KERNEL_KINDS = ("reduce", "prefilter", "stats", "calibrate", "shift", "combine")

c_p = ctypes.c_void_p
c_i = ctypes.c_int
c_i64 = ctypes.c_int64
c_sz = ctypes.c_size_t


class IrpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {STATUS_NAMES.get(self.status, self.status)}")


class ClipParams(ctypes.Structure):
    _fields_ = [("kappa_lo", ctypes.c_float), ("kappa_hi", ctypes.c_float),
                ("max_iter", c_i), ("center", c_i), ("ddof", c_i)]


class IrpSet(ctypes.Structure):
    _fields_ = [("frames", ctypes.POINTER(c_p)), ("raw_pitch", c_i64),
                ("W", c_i), ("H", c_i), ("n", c_i),
                ("dx", ctypes.POINTER(ctypes.c_double)), ("dy", ctypes.POINTER(ctypes.c_double)),
                ("exptime", ctypes.POINTER(ctypes.c_float)),
                ("bias", c_p), ("dark_rate", c_p), ("flat", c_p), ("master_pitch", c_i64),
                ("mean_out", c_p), ("median_out", c_p), ("nkept_out", c_p), ("out_pitch", c_i64),
                ("stack_out", c_p), ("ready_flag", c_p), ("ready_value", ctypes.c_uint32),
                ("mask", c_p), ("mask_pitch", c_i64), ("saturation", ctypes.c_float)]


class IrpHostIo(ctypes.Structure):
    _fields_ = [("frames", ctypes.POINTER(c_p)), ("pitch", c_i64), ("mean", c_p),
                ("median", c_p), ("nkept", c_p), ("out_pitch", c_i64)]


class ReduceParams(ctypes.Structure):
    _fields_ = [("interp", c_i), ("clip", ClipParams), ("normalize_flat", c_i),
                ("persistent", c_i), ("max_ctas", c_i), ("wait_spin_limit", c_i),
                ("rows_per_warp", c_i), ("frame_norm", c_i), ("spline_onchip", c_i)]


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Loads libirp.so (built by ``build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                                   "(run __graft_entry__.build() or python -m "
                                   "paper_2008_11486_gb300.build)")
            L = ctypes.CDLL(LIB_PATH)
            P, PP = ctypes.POINTER, c_p
            L.irp_version.restype = c_i
            L.irp_version.argtypes = []
            L.irp_status_string.restype = ctypes.c_char_p
            L.irp_status_string.argtypes = [c_i]
            L.irp_device_sm_count.restype = c_i
            L.irp_device_sm_count.argtypes = []
            L.irp_calibrate.restype = c_i
            L.irp_calibrate.argtypes = [PP, c_i64, c_i64, c_i, c_i, c_i, PP, PP, PP, c_i64,
                                        P(ctypes.c_float), c_i, PP, c_i64, c_i64, c_i, PP, PP,
                                        PP, c_sz, PP]
            L.irp_calibrate_workspace_size.restype = c_sz
            L.irp_calibrate_workspace_size.argtypes = [c_i]
            L.irp_frame_stats.restype = c_i
            L.irp_frame_stats.argtypes = [PP, c_i64, c_i64, c_i, c_i, c_i, c_i, PP, PP, PP, PP,
                                          PP, PP]
            L.irp_shift.restype = c_i
            L.irp_shift.argtypes = [PP, c_i64, c_i64, c_i, c_i, c_i, c_i, PP, PP,
                                    P(ctypes.c_double), P(ctypes.c_double), c_i, PP, c_i64,
                                    c_i64, PP, PP, c_sz, PP]
            L.irp_shift_workspace_size.restype = c_sz
            L.irp_shift_workspace_size.argtypes = [c_i, c_i, c_i, c_i]
            L.irp_combine.restype = c_i
            L.irp_combine.argtypes = [PP, c_i64, c_i64, c_i, c_i, c_i, c_i, PP, PP, PP,
                                      P(ClipParams), PP, PP, PP, PP, c_i64, PP]
            L.irp_workspace_size.restype = c_sz
            L.irp_workspace_size.argtypes = [P(IrpSet), c_i, P(ReduceParams)]
            L.irp_reduce_set.restype = c_i
            L.irp_reduce_set.argtypes = [P(IrpSet), c_i, P(ReduceParams), PP, c_sz, PP]
            L.irp_reduce_set_host.restype = c_i
            L.irp_reduce_set_host.argtypes = [P(IrpSet), c_i, P(IrpHostIo), P(ReduceParams),
                                              PP, c_sz, PP]
            L.irp_plan_bytes.restype = c_sz
            L.irp_plan_bytes.argtypes = [P(IrpSet), c_i, P(ReduceParams)]
            L.irp_plan_encode.restype = c_i
            L.irp_plan_encode.argtypes = [P(IrpSet), c_i, P(ReduceParams), PP, c_sz, PP, c_sz]
            L.irp_plan_launch.restype = c_i
            L.irp_plan_launch.argtypes = [PP, c_sz, PP, c_sz, PP]
            L.irp_sync_status.restype = c_i
            L.irp_sync_status.argtypes = [PP, PP]
            L.irp_last_cuda_error.restype = ctypes.c_char_p
            L.irp_last_cuda_error.argtypes = []
            L.irp_profile_enable.restype = None
            L.irp_profile_enable.argtypes = [c_i]
            L.irp_profile_read.restype = c_i
            L.irp_profile_read.argtypes = [PP, PP, c_i]
            _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != IRP_OK:
        if status == 6:
            where = f"{where} [{lib().irp_last_cuda_error().decode()}]"
        raise IrpError(status, where)
