"""GB300 GPU virtualization manager: Python binding of libgvm.

The method (Li, Narayana, El-Ghazawi, "Efficient Resource Sharing Through GPU
Virtualization on Accelerated High Performance Computing Systems"): many SPMD
ranks share one GPU through a single manager that owns the only context and
runs every rank's task -- input copy, kernel, output copy -- concurrently
(Section 4.2.2, Section 5). The compute and the scheduling run in the CUDA
library ``_build/libgvm.so`` (C ABI in ``include/gvm.h``); this module only
marshals arguments. PyTorch supplies device memory and streams.

Entry points: ``Manager`` (one manager; modes "barrier", "continuous",
"ps1", "ps2"; ``attach`` gives a ``Rank`` with ``submit_vadd``,
``submit_vmul``, ``submit_sgemm``, their resident forms, ``sync``, ``poll``;
``spmd_run``, ``spmd_run_overlapped`` and ``open_loop_run`` drive many ranks
from native threads), ``IpcRegion`` / ``IpcServer`` / ``IpcClient`` (ranks
in separate processes through shared memory), and the task kernels alone
(``vadd_f32``, ``vmul_f32``, ``sgemm_f32``).

There is no fallback: if the library is missing or no GPU is present, the
calls raise.
"""
from __future__ import annotations

import os

# More hardware queues than the default 8, so that the per-rank copy streams
# do not share queues (only effective before CUDA is initialised).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from ._abi import (  # noqa: E402
    GVM_EAGAIN,
    GVM_EBUSY,
    GVM_ECANCELED,
    GVM_EDEVICE,
    GVM_EINVAL,
    GVM_ENODEV,
    GVM_ENOMEM,
    GVM_ESTATE,
    GVM_ETIMEDOUT,
    GVM_IPC_ATTACHED,
    GVM_IPC_CLOSED,
    GVM_IPC_FREE,
    GVM_IPC_LOST,
    GVM_MODE_BARRIER,
    GVM_MODE_CONTINUOUS,
    GVM_MODE_PS1,
    GVM_MODE_PS2,
    GVM_OK,
    GVM_SGEMM_FMA,
    GVM_SGEMM_SPLIT3,
    GVM_TASK_RESIDENT,
    GVM_TASK_SGEMM,
    GVM_TASK_VADD,
    GVM_TASK_VMUL,
    GvmConfig,
    GvmError,
    GvmStats,
    GvmTask,
    lib,
    lib_path,
)
from .manager import Manager, Rank, sgemm_f32, sgemm_scratch_bytes, vadd_f32, vmul_f32  # noqa: E402
from .ipc import IpcClient, IpcRegion, IpcServer  # noqa: E402

__all__ = [
    "Manager",
    "Rank",
    "IpcRegion",
    "IpcServer",
    "IpcClient",
    "vadd_f32",
    "vmul_f32",
    "sgemm_f32",
    "sgemm_scratch_bytes",
    "lib",
    "lib_path",
    "GvmConfig",
    "GvmTask",
    "GvmStats",
    "GvmError",
    "GVM_OK",
    "GVM_EINVAL",
    "GVM_EBUSY",
    "GVM_EAGAIN",
    "GVM_ENOMEM",
    "GVM_ETIMEDOUT",
    "GVM_EDEVICE",
    "GVM_ECANCELED",
    "GVM_ESTATE",
    "GVM_ENODEV",
    "GVM_TASK_VADD",
    "GVM_TASK_SGEMM",
    "GVM_TASK_VMUL",
    "GVM_IPC_FREE",
    "GVM_IPC_ATTACHED",
    "GVM_IPC_CLOSED",
    "GVM_IPC_LOST",
    "GVM_TASK_RESIDENT",
    "GVM_SGEMM_FMA",
    "GVM_SGEMM_SPLIT3",
    "GVM_MODE_BARRIER",
    "GVM_MODE_CONTINUOUS",
    "GVM_MODE_PS1",
    "GVM_MODE_PS2",
]
