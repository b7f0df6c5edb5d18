"""ctypes declarations of the C ABI in include/gvm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading
from ctypes import POINTER, c_char_p, c_double, c_float, c_int, c_int32, c_int64, c_uint32, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
_DEFAULT_LIB = os.path.join(HERE, "_build", "libgvm.so")

GVM_OK = 0
GVM_EINVAL = -1
GVM_EBUSY = -2
GVM_EAGAIN = -3
GVM_ENOMEM = -4
GVM_ETIMEDOUT = -5
GVM_EDEVICE = -6
GVM_ECANCELED = -7
GVM_ESTATE = -8
GVM_ENODEV = -9

GVM_TASK_VADD = 1
GVM_TASK_SGEMM = 2
GVM_TASK_VMUL = 3
GVM_TASK_RESIDENT = 1
GVM_SGEMM_FMA = 0
GVM_SGEMM_SPLIT3 = 1
GVM_SGEMM_SPLIT3_FUSED = 2
GVM_SGEMM_SPLIT3_WIDE = 4
GVM_SGEMM_SPLIT3_TMA = 5
GVM_MODE_BARRIER = 0
GVM_MODE_CONTINUOUS = 1
GVM_MODE_PS1 = 2
GVM_MODE_PS2 = 3


class GvmConfig(ctypes.Structure):
    _fields_ = [
        ("max_ranks", c_int32),
        ("ring_depth", c_int32),
        ("mode", c_int32),
        ("sgemm_path", c_int32),
        ("arena", c_void_p),
        ("arena_bytes", c_uint64),
        ("resident_bytes", c_uint64),
        ("ctrl", c_void_p),
        ("ctrl_bytes", c_uint64),
        ("sched_stream", c_void_p),
        ("copy_streams", POINTER(c_void_p)),
        ("admission_cap_bytes", c_uint64),
        ("wait_timeout_ns", c_uint64),
        ("idle_poll_ns", c_uint64),
        ("grid_ctas", c_int32),
        ("ingest_quantum", c_int32),
        ("copy_run_bytes", c_uint64),
        ("vadd_tile", c_int64),
        ("direct_output", c_int32),
        ("l2_prefetch", c_int32),
        ("copy_streams_max", c_int32),
        ("copy_in_streams", c_int32),
    ]


class GvmTask(ctypes.Structure):
    _fields_ = [
        ("type", c_int32),
        ("flags", c_int32),
        ("n", c_int64),
        ("m", c_int32),
        ("k", c_int32),
        ("a", c_void_p),
        ("b", c_void_p),
        ("c", c_void_p),
        ("a_off", c_uint64),
        ("b_off", c_uint64),
        ("c_off", c_uint64),
    ]


class GvmStats(ctypes.Structure):
    _fields_ = [
        ("submitted", c_uint64),
        ("completed", c_uint64),
        ("launches", c_uint64),
        ("staged_bytes", c_uint64),
        ("staged_peak", c_uint64),
        ("h2d_bytes", c_uint64),
        ("d2h_bytes", c_uint64),
        ("device_status", c_uint32),
        ("device_where", c_uint32),
        ("launch_start_ns", c_uint64),
        ("launch_last_done_ns", c_uint64),
        ("launch_exit_ns", c_uint64),
        ("launch_phase", c_uint64 * 12),
    ]


class GvmIpcTask(ctypes.Structure):
    """gvm_ipc_task: one cross-process request (offsets into the rank's data area)."""

    _fields_ = [
        ("type", c_int32),
        ("reserved", c_int32),
        ("m", c_int64),
        ("n", c_int64),
        ("k", c_int64),
        ("a_off", c_uint64),
        ("b_off", c_uint64),
        ("c_off", c_uint64),
    ]


GVM_IPC_FREE = 0
GVM_IPC_ATTACHED = 1
GVM_IPC_CLOSED = 2
GVM_IPC_LOST = 3


class GvmError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = lib().gvm_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


# name -> (restype, argtypes)
PROTOTYPES = {
    "gvm_ctrl_bytes": (c_uint64, [POINTER(GvmConfig)]),
    "gvm_init": (c_int, [POINTER(GvmConfig), POINTER(c_void_p)]),
    "gvm_attach": (c_int, [c_void_p, c_int32, POINTER(c_void_p)]),
    "gvm_submit": (c_int, [c_void_p, POINTER(GvmTask), POINTER(c_uint64)]),
    "gvm_submit_many": (c_int, [c_void_p, POINTER(GvmTask), c_uint32, POINTER(c_uint64)]),
    "gvm_sync": (c_int, [c_void_p, c_uint64]),
    "gvm_poll": (c_int, [c_void_p, c_uint64]),
    "gvm_flush": (c_int, [c_void_p]),
    "gvm_wait_idle": (c_int, [c_void_p]),
    "gvm_rank_write": (c_int, [c_void_p, c_uint64, c_void_p, c_uint64]),
    "gvm_rank_read": (c_int, [c_void_p, c_uint64, c_void_p, c_uint64]),
    "gvm_rank_resident_ptr": (c_void_p, [c_void_p]),
    "gvm_stream": (c_void_p, [c_void_p, c_int32]),
    "gvm_detach": (c_int, [c_void_p]),
    "gvm_shutdown": (c_int, [c_void_p]),
    "gvm_stats_get": (c_int, [c_void_p, POINTER(GvmStats)]),
    "gvm_task_times": (c_int, [c_void_p, c_uint64, POINTER(c_uint64), POINTER(c_uint64)]),
    "gvm_spmd_run": (
        c_int,
        [c_void_p, POINTER(c_void_p), POINTER(POINTER(GvmTask)), POINTER(c_uint32), c_int32, c_int32,
         POINTER(c_float), POINTER(c_float), POINTER(c_double), POINTER(POINTER(c_double))],
    ),
    "gvm_spmd_run_overlapped": (
        c_int,
        [c_void_p, POINTER(c_void_p), POINTER(POINTER(GvmTask)), POINTER(POINTER(GvmTask)), POINTER(c_uint32),
         c_int32, c_int32, POINTER(c_double), POINTER(c_double)],
    ),
    "gvm_spmd_run_pipelined": (
        c_int,
        [c_void_p, POINTER(c_void_p), POINTER(POINTER(POINTER(GvmTask))), c_int32, POINTER(c_uint32), c_int32,
         c_int32, POINTER(c_double), POINTER(c_double)],
    ),
    "gvm_open_loop_run": (
        c_int,
        [c_void_p, POINTER(c_void_p), POINTER(POINTER(GvmTask)), POINTER(POINTER(c_uint64)), POINTER(c_uint32),
         c_int32, c_uint32, POINTER(POINTER(c_double)), POINTER(c_double)],
    ),
    "gvm_strerror": (c_char_p, [c_int]),
    "gvm_vadd_f32": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p]),
    "gvm_vmul_f32": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_void_p]),
    "gvm_sgemm_scratch_bytes": (c_uint64, [c_int32, c_int32, c_int32, c_int32]),
    "gvm_sgemm_f32": (
        c_int,
        [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p, c_uint64, c_void_p],
    ),
    "gvm_kernel_status": (c_int, [POINTER(c_uint32)]),
    "gvm_sgemm_f32_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_void_p]),
    # cross-process ranks (gvm_ipc.h)
    "gvm_ipc_create": (c_int, [c_char_p, c_int32, c_uint64, c_int32, POINTER(c_void_p)]),
    "gvm_ipc_destroy": (c_int, [c_void_p]),
    "gvm_ipc_serve": (c_int, [c_void_p, c_void_p, POINTER(c_void_p)]),
    "gvm_ipc_stop": (c_int, [c_void_p]),
    "gvm_ipc_server_counts": (c_int, [c_void_p, POINTER(c_uint64), POINTER(c_uint64), POINTER(c_uint64)]),
    "gvm_ipc_peek": (
        c_int, [c_void_p, c_int32, POINTER(c_uint64), POINTER(c_uint64), POINTER(c_uint64), POINTER(c_uint32)]
    ),
    "gvm_ipc_open": (c_int, [c_char_p, c_int32, POINTER(c_void_p)]),
    "gvm_ipc_data": (c_void_p, [c_void_p, POINTER(c_uint64)]),
    "gvm_ipc_submit": (c_int, [c_void_p, POINTER(GvmIpcTask), POINTER(c_uint64)]),
    "gvm_ipc_barrier": (c_int, [c_void_p]),
    "gvm_ipc_wait": (c_int, [c_void_p, c_uint64, c_uint64]),
    "gvm_ipc_close": (c_int, [c_void_p]),
}

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return os.environ.get("GVM_LIB", _DEFAULT_LIB)


def lib():
    """The loaded libgvm.so. Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    f"libgvm.so not found at {path}; build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`"
                )
            handle = ctypes.CDLL(path)
            for name, (res, args) in PROTOTYPES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def check(code: int, what: str = "") -> int:
    if code < 0:
        raise GvmError(code, what)
    return code
