"""Cross-process ranks (include/gvm_ipc.h): argument marshalling only.

Manager process::

    region = IpcRegion.create("job42", nranks=16, data_bytes=256 << 20)
    with Manager(16, mode="barrier") as mgr:
        server = IpcServer(mgr, region)
        ...                       # clients run in their own processes
        server.stop()
    region.destroy()

Client process (no CUDA)::

    c = IpcClient("job42", rank)
    x = c.floats(0, n); y = c.floats(4 * n, n)      # views of the data area
    seq = c.submit_vadd(0, 4 * n, 8 * n, n)
    c.barrier(); c.wait(seq)
    c.close()

Each rank's segment is its own POSIX shared-memory object; a client maps
only its own (Section 5's per-process shared data, with the operating system
keeping ranks apart).
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_uint32, c_uint64, c_void_p

import numpy as np

from ._abi import (
    GVM_IPC_ATTACHED,
    GVM_IPC_CLOSED,
    GVM_IPC_FREE,
    GVM_IPC_LOST,
    GVM_TASK_SGEMM,
    GVM_TASK_VADD,
    GVM_TASK_VMUL,
    GvmIpcTask,
    check,
    lib,
)

__all__ = [
    "IpcRegion",
    "IpcServer",
    "IpcClient",
    "GVM_IPC_FREE",
    "GVM_IPC_ATTACHED",
    "GVM_IPC_CLOSED",
    "GVM_IPC_LOST",
]


class IpcRegion:
    """The per-rank shared-memory segments (manager side)."""

    def __init__(self, handle: int, name: str, nranks: int):
        self.handle = handle
        self.name = name
        self.nranks = nranks

    @classmethod
    def create(cls, name: str, nranks: int, data_bytes: int, depth: int = 64) -> "IpcRegion":
        h = c_void_p()
        check(lib().gvm_ipc_create(name.encode(), nranks, data_bytes, depth, byref(h)), "gvm_ipc_create")
        return cls(h.value, name, nranks)

    def peek(self, rank: int) -> dict:
        head, arrived, done, state = c_uint64(), c_uint64(), c_uint64(), c_uint32()
        check(lib().gvm_ipc_peek(self.handle, rank, byref(head), byref(arrived), byref(done), byref(state)),
              "gvm_ipc_peek")
        return {"head": head.value, "arrived": arrived.value, "done": done.value, "state": state.value}

    def destroy(self) -> None:
        if self.handle is not None:
            check(lib().gvm_ipc_destroy(self.handle), "gvm_ipc_destroy")
            self.handle = None


class IpcServer:
    """The manager's serving thread for a region (ranks 0..nranks-1 of mgr)."""

    def __init__(self, mgr, region: IpcRegion):
        h = c_void_p()
        check(lib().gvm_ipc_serve(mgr.handle, region.handle, byref(h)), "gvm_ipc_serve")
        self.handle = h.value

    def counts(self) -> dict:
        t, c, b = c_uint64(), c_uint64(), c_uint64()
        check(lib().gvm_ipc_server_counts(self.handle, byref(t), byref(c), byref(b)), "gvm_ipc_server_counts")
        return {"taken": t.value, "completed": c.value, "barriers": b.value}

    def stop(self) -> None:
        if self.handle is not None:
            h, self.handle = self.handle, None
            check(lib().gvm_ipc_stop(h), "gvm_ipc_stop")


class IpcClient:
    """One rank's mapping of its segment (client side; no CUDA call)."""

    def __init__(self, name: str, rank: int):
        h = c_void_p()
        check(lib().gvm_ipc_open(name.encode(), rank, byref(h)), "gvm_ipc_open")
        self.handle = h.value
        nb = c_uint64()
        ptr = lib().gvm_ipc_data(self.handle, byref(nb))
        self.data_bytes = nb.value
        self._buf = (ctypes.c_uint8 * nb.value).from_address(ptr)
        self.data = np.frombuffer(self._buf, dtype=np.uint8)

    def floats(self, off: int, count: int) -> np.ndarray:
        """A float32 view of `count` values at byte offset `off` of the data area."""
        return self.data[off : off + 4 * count].view(np.float32)

    def submit(self, type_: int, *, m: int = 0, n: int = 0, k: int = 0, a_off: int = 0, b_off: int = 0,
               c_off: int = 0) -> int:
        t = GvmIpcTask()
        t.type, t.reserved = type_, 0
        t.m, t.n, t.k = m, n, k
        t.a_off, t.b_off, t.c_off = a_off, b_off, c_off
        seq = c_uint64()
        check(lib().gvm_ipc_submit(self.handle, byref(t), byref(seq)), "gvm_ipc_submit")
        return seq.value

    def submit_vadd(self, a_off: int, b_off: int, c_off: int, n: int) -> int:
        return self.submit(GVM_TASK_VADD, n=n, a_off=a_off, b_off=b_off, c_off=c_off)

    def submit_vmul(self, a_off: int, b_off: int, c_off: int, n: int, iters: int) -> int:
        return self.submit(GVM_TASK_VMUL, n=n, k=iters, a_off=a_off, b_off=b_off, c_off=c_off)

    def submit_sgemm(self, a_off: int, b_off: int, c_off: int, m: int, n: int, k: int) -> int:
        return self.submit(GVM_TASK_SGEMM, m=m, n=n, k=k, a_off=a_off, b_off=b_off, c_off=c_off)

    def barrier(self) -> None:
        check(lib().gvm_ipc_barrier(self.handle), "gvm_ipc_barrier")

    def wait(self, seq: int, timeout_s: float = 0.0) -> None:
        check(lib().gvm_ipc_wait(self.handle, seq, int(timeout_s * 1e9)), "gvm_ipc_wait")

    def wait_code(self, seq: int, timeout_s: float = 0.0) -> int:
        """gvm_ipc_wait's return code (0 or a negative GVM_* error)."""
        return lib().gvm_ipc_wait(self.handle, seq, int(timeout_s * 1e9))

    def close(self) -> None:
        if self.handle is not None:
            self.data = None
            self._buf = None
            h, self.handle = self.handle, None
            check(lib().gvm_ipc_close(h), "gvm_ipc_close")
