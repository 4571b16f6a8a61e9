"""ctypes declarations of the LINVIEW C ABI (include/linview.h).

Loading fails loudly: there is no Python or CPU implementation behind these
names, only the CUDA library built from ``csrc/``.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblinview.so")

# linview_status
OK, EINVAL, ESHAPE, ENOMEM, ERANK, ESINGULAR, ENONFINITE, ETIMEOUT, EDEVICE, EUNSUPPORTED = range(10)
STATUS_NAMES = ["OK", "EINVAL", "ESHAPE", "ENOMEM", "ERANK", "ESINGULAR", "ENONFINITE",
                "ETIMEOUT", "EDEVICE", "EUNSUPPORTED"]
# linview_kind
POWER, POWER_SUM, ITERATION, OLS = range(4)
# linview_precision
F64, F32 = 0, 1
# linview_reeval_mode
REEVAL_DEFAULT, REEVAL_FP32, REEVAL_TF32, REEVAL_BF16X9, REEVAL_FP64, REEVAL_TC3 = range(6)
# linview_model
MODEL_EXP, MODEL_LINEAR, MODEL_SKIP = 0, 1, 2
STRATEGY_FACTORED, STRATEGY_HYBRID = 0, 1
# linview_correction
CORRECT_REEVAL, CORRECT_NEWTON = 0, 1
DST_HOST, DST_DEVICE, DST_HOST_ASYNC = 0, 1, 2  # read destinations


class ProgramDesc(C.Structure):
    _fields_ = [
        ("kind", C.c_int32),
        ("precision", C.c_int32),
        ("n", C.c_int64),
        ("m", C.c_int64),
        ("p", C.c_int64),
        ("k", C.c_int32),
        ("r_max", C.c_int32),
        ("correction_period", C.c_int32),
        ("reeval_mode", C.c_int32),
        ("model", C.c_int32),
        ("skip", C.c_int32),
        ("strategy", C.c_int32),
        ("alloc", C.c_void_p),
        ("free", C.c_void_p),
        ("alloc_ctx", C.c_void_p),
        ("correction", C.c_int32),
    ]


# device-memory callbacks of linview_program_desc
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Completion(C.Structure):
    _fields_ = [
        ("ticket", C.c_uint64),
        ("view", C.c_int32),
        ("rank", C.c_int32),
        ("batch_rank", C.c_int32),
        ("batch_size", C.c_int32),
        ("status", C.c_int32),
        ("reserved", C.c_int32),
        ("arrival_s", C.c_double),
        ("start_s", C.c_double),
        ("done_s", C.c_double),
    ]


class ServerStats(C.Structure):
    _fields_ = [
        ("submitted", C.c_int64),
        ("completed", C.c_int64),
        ("failed", C.c_int64),
        ("refreshes", C.c_int64),
        ("coalesced_rank_sum", C.c_int64),
        ("views_resident", C.c_int32),
        ("views_waiting", C.c_int32),
        ("max_inflight_seen", C.c_int32),
        ("reevals", C.c_int32),
        ("bytes_used", C.c_int64),
        ("bytes_budget", C.c_int64),
    ]


class LinviewError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{fn} -> {name}: {msg}")
        self.status = status
        self.name = name


_P = C.c_void_p
_I64 = C.c_int64
_I = C.c_int

# (name, restype, argtypes); the status-returning calls are checked
_SIGS = [
    ("linview_create_program", _I, [C.POINTER(ProgramDesc), C.POINTER(_P), C.POINTER(_I64), _I, _P,
                                    C.POINTER(_P)]),
    ("linview_apply_delta", _I, [_P, _I, _I64, _P, _I64, _P, _I64, _I, _P]),
    ("linview_apply_row_delta", _I, [_P, _I, _I64, _P, _I, _P]),
    ("linview_apply_row_block", _I, [_P, _I64, C.POINTER(_I64), _P, _I64, _I, _P]),
    ("linview_num_views", _I, [_P]),
    ("linview_view_shape", _I, [_P, _I, C.POINTER(_I64), C.POINTER(_I64)]),
    ("linview_read_view", _I, [_P, _I, _P, _I64, _I, _P]),
    ("linview_read_view_rows", _I, [_P, _I, _I64, _I64, _P, _I64, _I, _P]),
    ("linview_view_device_ptr", _I, [_P, _I, C.POINTER(_P), C.POINTER(_I64)]),
    ("linview_reeval", _I, [_P, _P]),
    ("linview_correct", _I, [_P, _P]),
    ("linview_set_reeval_mode", _I, [_P, _I]),
    ("linview_sync", _I, [_P, _P]),
    ("linview_prepare_updates", _I, [_P, _I, _P]),
    ("linview_check_bounded_wait", _I, [_I64, _P, C.POINTER(_I64)]),
    ("linview_destroy", None, [_P]),
    ("linview_last_error", C.c_char_p, []),
    ("linview_adjoint_iteration", _I, [_P, _P, _I64, _P, _I64, _P]),
    ("linview_adjoint_iteration_seed", _I, [_P, _P, _I64, _P, _I64, _P, _I64, _P, _I64, _P]),
    ("linview_adjoint_power", _I, [_P, _P, _I64, _P, _I64, _P]),
    ("linview_gemm", _I, [_I, _I, _I, _I64, _I64, _I64, C.c_double, _P, _I64, _P, _I64,
                          C.c_double, _P, _I64, _P]),
    ("linview_level_pass", _I, [_I, _I64, _P, _I64, _P, _P, _I64, _I64, _P, _P, _I, _P]),
    ("linview_level_pass_noalloc", _I, [_I, _I64, _P, _I64, _P, _P, _I64, _I64, _P, _P, _I, _P]),
    ("linview_set_profiling", _I, [_P, _I]),
    ("linview_pass_stats", _I, [_P, _I, C.POINTER(_I64), C.POINTER(C.c_double),
                                C.POINTER(C.c_double), C.POINTER(_I64)]),
    ("linview_reset_stats", _I, [_P]),
    ("linview_program_device_bytes", _I, [_P, C.POINTER(_I64)]),
    ("linview_estimate_device_bytes", _I, [C.POINTER(ProgramDesc), C.POINTER(_I64)]),
    ("linview_server_create", _I, [_I64, C.c_int32, C.c_int32, C.POINTER(_P)]),
    ("linview_server_add_view", _I, [_P, _I64, C.c_int32, _P, _I64, _I, C.POINTER(C.c_int32)]),
    ("linview_server_submit", _I, [_P, C.c_int32, C.c_int32, _P, _I64, _P, _I64, C.c_double,
                                   C.POINTER(C.c_uint64)]),
    ("linview_server_submit_row", _I, [_P, C.c_int32, _I64, _P, C.c_double,
                                       C.POINTER(C.c_uint64)]),
    ("linview_server_replay", _I, [_P, _I64, _P, _P, _P, _P, _P, _P]),
    ("linview_server_poll", _I, [_P, _P, C.c_int32, C.POINTER(C.c_int32)]),
    ("linview_server_drain", _I, [_P, C.c_double]),
    ("linview_server_view_state", _I, [_P, C.c_int32, C.POINTER(C.c_int32)]),
    ("linview_server_view_program", _I, [_P, C.c_int32, C.POINTER(_P)]),
    ("linview_server_remove_view", _I, [_P, C.c_int32]),
    ("linview_server_stats_get", _I, [_P, _P]),
    ("linview_server_clock", C.c_double, [_P]),
    ("linview_server_destroy", None, [_P]),
]

EXPORTED = [s[0] for s in _SIGS]
_lib = None


def load(path: str = LIB_PATH):
    """Load liblinview.so (raise if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with `python -m paper_1403_6968_gb300.build` "
            "(needs nvcc; there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, fn: str):
    if status != OK:
        msg = load().linview_last_error()
        raise LinviewError(status, fn, msg.decode() if msg else "")


def call(name: str, *args):
    """Call a status-returning ABI function and raise on error."""
    st = getattr(load(), name)(*args)
    check(st, name)
    return st
