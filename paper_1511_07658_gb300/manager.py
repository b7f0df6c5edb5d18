"""Thin Python wrappers over the gvm C ABI.

``Manager`` allocates the device arena and control block with PyTorch and
passes raw pointers to ``gvm_init`` (which creates the streams). ``Rank``
wraps a rank handle (the paper's virtual GPU, Section 5): ``submit_*`` is
SND()+STR(), ``sync`` is STP()+RCV(). Every step of a task runs in libgvm.
"""
from __future__ import annotations

import ctypes
import json
import os
from ctypes import byref, c_uint32, c_uint64, c_void_p

import torch

from . import _abi
from ._abi import (
    GVM_EAGAIN,
    GVM_MODE_BARRIER,
    GVM_MODE_CONTINUOUS,
    GVM_MODE_PS1,
    GVM_MODE_PS2,
    GVM_SGEMM_FMA,
    GVM_SGEMM_SPLIT3,
    GVM_SGEMM_SPLIT3_FUSED,
    GVM_SGEMM_SPLIT3_TMA,
    GVM_SGEMM_SPLIT3_WIDE,
    GVM_TASK_RESIDENT,
    GVM_TASK_SGEMM,
    GVM_TASK_VADD,
    GVM_TASK_VMUL,
    GvmConfig,
    GvmStats,
    GvmTask,
    check,
    lib,
)

_PATHS = {
    "fma": GVM_SGEMM_FMA,
    "split3": GVM_SGEMM_SPLIT3,
    "split3_fused": GVM_SGEMM_SPLIT3_FUSED,
    "split3_wide": GVM_SGEMM_SPLIT3_WIDE,
    "split3_tma": GVM_SGEMM_SPLIT3_TMA,
}
_MODES = {"barrier": GVM_MODE_BARRIER, "continuous": GVM_MODE_CONTINUOUS, "ps1": GVM_MODE_PS1, "ps2": GVM_MODE_PS2}


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream_handle(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


TUNING_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def tuning() -> dict:
    """Manager parameters chosen by ``autotune`` on a GB300 (the committed
    table), or {} when there is none: the library's own defaults apply."""
    try:
        with open(TUNING_FILE) as f:
            return json.load(f).get("choice", {})
    except (OSError, ValueError):
        return {}


class Rank:
    """One rank's virtual GPU: its ring, arena slice and streams."""

    def __init__(self, mgr: "Manager", rank: int, handle: int):
        self.mgr = mgr
        self.rank = rank
        self.handle = c_void_p(handle)
        self.resident_bytes = mgr.resident_bytes

    # -- submission -------------------------------------------------------
    def submit(self, task: GvmTask, block: bool = True) -> int:
        """Submit a task; returns its sequence number. With ``block`` the call
        retries while the ring or staging space is full (syncing on the rank's
        oldest unfinished task), otherwise GVM_EAGAIN raises."""
        seq = c_uint64(0)
        L = lib()
        while True:
            rc = L.gvm_submit(self.handle, byref(task), byref(seq))
            if rc == GVM_EAGAIN and block:
                self.mgr.flush_if_barrier()
                self._sync_checked(self._oldest_pending())
                continue
            check(rc, "gvm_submit")
            self._last = seq.value
            return seq.value

    def submit_many(self, tasks, block: bool = True) -> tuple[int, int]:
        """Submit a ctypes array of GvmTask in order; returns (first_seq,
        count). With ``block`` a full ring or staging ring is waited out."""
        L = lib()
        first = c_uint64(0)
        total, first_seq = 0, None
        n = len(tasks)
        base = ctypes.addressof(tasks)
        size = ctypes.sizeof(GvmTask)
        while total < n:
            ptr = ctypes.cast(base + total * size, ctypes.POINTER(GvmTask))
            rc = L.gvm_submit_many(self.handle, ptr, n - total, byref(first))
            check(rc, "gvm_submit_many")
            if rc > 0:
                if first_seq is None:
                    first_seq = first.value
                total += rc
                self._last = first.value + rc - 1
            if total < n:
                if not block:
                    break
                self.mgr.flush_if_barrier()
                self._sync_checked(self._oldest_pending())
        return (first_seq if first_seq is not None else -1), total

    def _sync_checked(self, seq: int) -> None:
        rc = lib().gvm_sync(self.handle, seq)
        if rc != 0:
            st = self.mgr.stats()
            check(rc, f"gvm_sync (device status {st['device_status']}, where {st['device_where']})")

    def _oldest_pending(self) -> int:
        last = getattr(self, "_last", None)
        if last is None:
            return 0
        lo = max(0, last - self.mgr.ring_depth + 1)
        for s in range(lo, last + 1):
            if L_poll(self.handle, s) == 0:
                return s
        return last

    def submit_vadd(self, a: torch.Tensor, b: torch.Tensor, c: torch.Tensor, block: bool = True) -> int:
        """Host mode: a, b, c are pinned float32 host tensors of equal length."""
        t = GvmTask()
        t.type = GVM_TASK_VADD
        t.flags = 0
        t.n = a.numel()
        t.a, t.b, t.c = _ptr(a), _ptr(b), _ptr(c)
        return self.submit(t, block)

    def submit_vmul(self, a: torch.Tensor, b: torch.Tensor, c: torch.Tensor, iters: int, block: bool = True) -> int:
        """Host mode: c = a * b * ... * b with `iters` float32 products per element."""
        t = GvmTask()
        t.type = GVM_TASK_VMUL
        t.flags = 0
        t.n = a.numel()
        t.k = iters
        t.a, t.b, t.c = _ptr(a), _ptr(b), _ptr(c)
        return self.submit(t, block)

    def submit_sgemm(self, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, block: bool = True) -> int:
        """Host mode: pinned float32 host tensors A (m x k), B (k x n), C (m x n)."""
        t = GvmTask()
        t.type = GVM_TASK_SGEMM
        t.flags = 0
        t.m, t.k = A.shape
        t.n = B.shape[1]
        t.a, t.b, t.c = _ptr(A), _ptr(B), _ptr(C)
        return self.submit(t, block)

    def submit_vadd_resident(self, a_off: int, b_off: int, c_off: int, n: int, block: bool = True) -> int:
        t = GvmTask()
        t.type = GVM_TASK_VADD
        t.flags = GVM_TASK_RESIDENT
        t.n = n
        t.a_off, t.b_off, t.c_off = a_off, b_off, c_off
        return self.submit(t, block)

    def submit_vmul_resident(self, a_off: int, b_off: int, c_off: int, n: int, iters: int, block: bool = True) -> int:
        t = GvmTask()
        t.type = GVM_TASK_VMUL
        t.flags = GVM_TASK_RESIDENT
        t.n, t.k = n, iters
        t.a_off, t.b_off, t.c_off = a_off, b_off, c_off
        return self.submit(t, block)

    def submit_sgemm_resident(
        self, a_off: int, b_off: int, c_off: int, m: int, n: int, k: int, block: bool = True
    ) -> int:
        t = GvmTask()
        t.type = GVM_TASK_SGEMM
        t.flags = GVM_TASK_RESIDENT
        t.m, t.n, t.k = m, n, k
        t.a_off, t.b_off, t.c_off = a_off, b_off, c_off
        return self.submit(t, block)

    # -- completion -------------------------------------------------------
    def sync(self, seq: int) -> None:
        rc = lib().gvm_sync(self.handle, seq)
        if rc == _abi.GVM_EDEVICE and self.mgr.handle is not None:
            st = self.mgr.stats()
            check(rc, f"gvm_sync (device status {st['device_status']}, where {st['device_where']})")
        check(rc, "gvm_sync")

    def poll(self, seq: int) -> bool:
        return check(lib().gvm_poll(self.handle, seq), "gvm_poll") == 1

    def task_times(self, seq: int) -> tuple[int, int]:
        a, b = c_uint64(0), c_uint64(0)
        check(lib().gvm_task_times(self.handle, seq, byref(a), byref(b)), "gvm_task_times")
        return a.value, b.value

    # -- resident region --------------------------------------------------
    def write(self, off: int, src: torch.Tensor) -> None:
        check(lib().gvm_rank_write(self.handle, off, _ptr(src), src.numel() * src.element_size()), "gvm_rank_write")

    def read(self, off: int, dst: torch.Tensor) -> None:
        check(lib().gvm_rank_read(self.handle, off, _ptr(dst), dst.numel() * dst.element_size()), "gvm_rank_read")

    def resident_ptr(self) -> int:
        return lib().gvm_rank_resident_ptr(self.handle)

    def resident_view(self, off: int, shape, dtype=torch.float32) -> torch.Tensor:
        """A torch view of the rank's resident region (the region is a slice of
        the manager's torch arena)."""
        n = 1
        for s in shape:
            n *= s
        esz = torch.empty(0, dtype=dtype).element_size()
        base = self.resident_ptr() - self.mgr.arena.data_ptr() + off
        if off + n * esz > self.resident_bytes:
            raise ValueError("view exceeds the resident region")
        return self.mgr.arena[base : base + n * esz].view(dtype).view(*shape)

    def detach(self) -> None:
        check(lib().gvm_detach(self.handle), "gvm_detach")


def L_poll(handle, seq):
    return lib().gvm_poll(handle, seq)


class Manager:
    """One GPU virtualization manager on the current CUDA device."""

    def __init__(
        self,
        ranks: int,
        *,
        ring_depth: int = 64,
        mode: str = "barrier",
        sgemm_path: str | None = None,
        slice_bytes: int = 64 << 20,
        resident_bytes: int = 0,
        admission_cap_bytes: int = 0,
        wait_timeout_s: float = 10.0,
        idle_poll_ns: int = 1000,
        grid_ctas: int = 0,
        ingest_quantum: int = 4,
        copy_run_bytes: int | None = None,
        vadd_tile: int | None = None,
        direct_output: bool | None = None,
        l2_prefetch: bool | None = None,
        copy_streams_max: int = 0,
        copy_in_streams: int = 0,
        device: int | None = None,
    ):
        if not torch.cuda.is_available():
            raise RuntimeError("gvm Manager needs a CUDA device")
        L = lib()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.ranks = ranks
        self.ring_depth = ring_depth
        self.mode = mode
        self.resident_bytes = resident_bytes
        self.slice_bytes = slice_bytes
        cfg = GvmConfig()
        cfg.max_ranks = ranks
        cfg.ring_depth = ring_depth
        cfg.mode = _MODES[mode]
        if sgemm_path is None:  # the autotuner's form, else the fused split3 tiles
            sgemm_path = tuning().get("sgemm_form", "split3")
        cfg.sgemm_path = _PATHS[sgemm_path]
        ctrl_bytes = L.gvm_ctrl_bytes(byref(cfg))
        if ctrl_bytes == 0:
            raise ValueError("invalid manager configuration")
        with torch.cuda.device(self.device):
            self.arena = torch.empty(slice_bytes * ranks + 256, dtype=torch.uint8, device=self.device)
            self.ctrl = torch.empty(ctrl_bytes + 256, dtype=torch.uint8, device=self.device)
        arena_ptr = (self.arena.data_ptr() + 255) // 256 * 256
        ctrl_ptr = (self.ctrl.data_ptr() + 255) // 256 * 256
        cfg.arena = arena_ptr
        cfg.arena_bytes = slice_bytes * ranks
        cfg.resident_bytes = resident_bytes
        cfg.ctrl = ctrl_ptr
        cfg.ctrl_bytes = ctrl_bytes
        # Streams: the manager creates dedicated non-blocking ones (PyTorch's
        # stream pool recycles a fixed set, so two pool streams can alias).
        cfg.sched_stream = None
        cfg.copy_streams = None
        cfg.admission_cap_bytes = admission_cap_bytes
        cfg.wait_timeout_ns = int(wait_timeout_s * 1e9)
        cfg.idle_poll_ns = idle_poll_ns
        cfg.grid_ctas = grid_ctas
        cfg.ingest_quantum = ingest_quantum
        tuned = tuning()
        cfg.copy_run_bytes = int(tuned.get("copy_run_bytes", 0) if copy_run_bytes is None else copy_run_bytes)
        cfg.vadd_tile = int(tuned.get("vadd_tile", 0) if vadd_tile is None else vadd_tile)
        cfg.direct_output = int(bool(tuned.get("direct_output", 0) if direct_output is None else direct_output))
        cfg.l2_prefetch = int(bool(tuned.get("l2_prefetch", 0) if l2_prefetch is None else l2_prefetch))
        cfg.copy_streams_max = int(copy_streams_max)
        cfg.copy_in_streams = int(copy_in_streams)
        self.cfg = cfg
        h = c_void_p()
        with torch.cuda.device(self.device):
            check(L.gvm_init(byref(cfg), byref(h)), "gvm_init")
        self.handle = h
        self._ranks: dict[int, Rank] = {}
        # PyTorch views of the manager's streams, for events and for queueing
        # work on them; valid until shutdown.
        self.sched_stream = torch.cuda.ExternalStream(L.gvm_stream(h, -1), device=self.device)
        self.copy_streams = [
            torch.cuda.ExternalStream(L.gvm_stream(h, i), device=self.device) for i in range(2 * ranks)
        ]

    def attach(self, rank: int) -> Rank:
        h = c_void_p()
        check(lib().gvm_attach(self.handle, rank, byref(h)), "gvm_attach")
        r = Rank(self, rank, h.value)
        self._ranks[rank] = r
        return r

    def flush(self) -> None:
        check(lib().gvm_flush(self.handle), "gvm_flush")

    def flush_if_barrier(self) -> None:
        """gvm_flush in every mode that needs one (all but continuous)."""
        if self.mode != "continuous":
            self.flush()

    def wait_idle(self) -> None:
        check(lib().gvm_wait_idle(self.handle), "gvm_wait_idle")

    def stats(self) -> dict:
        s = GvmStats()
        check(lib().gvm_stats_get(self.handle, byref(s)), "gvm_stats_get")
        out = {name: getattr(s, name) for name, _ in GvmStats._fields_}
        out["launch_phase"] = list(s.launch_phase)
        return out

    def spmd_run(self, ranks, task_arrays, steps: int, latency: bool = False):
        """Runs ``steps`` SPMD steps natively (gvm_spmd_run): one thread per
        rank submits ``task_arrays[i]`` (a ctypes array of GvmTask) for
        ``ranks[i]``, then flush and sync. Returns per-step times in ms:
        (step, scheduler launch) by CUDA events on the scheduler stream, and
        the step on the host clock. With ``latency``, a fourth item: per rank,
        the host-clock latency in seconds of every task of every step, from
        the rank's submit call to the moment the rank saw it complete."""
        n = len(ranks)
        hs = (c_void_p * n)(*[r.handle for r in ranks])
        tp = (ctypes.POINTER(GvmTask) * n)(*[ctypes.cast(a, ctypes.POINTER(GvmTask)) for a in task_arrays])
        cnt = (c_uint32 * n)(*[len(a) for a in task_arrays])
        dev = (ctypes.c_float * max(steps, 1))()
        launch = (ctypes.c_float * max(steps, 1))()
        host = (ctypes.c_double * max(steps, 1))()
        lat = lp = None
        if latency:
            lat = [(ctypes.c_double * max(steps * len(a), 1))() for a in task_arrays]
            lp = (ctypes.POINTER(ctypes.c_double) * n)(*[ctypes.cast(x, ctypes.POINTER(ctypes.c_double)) for x in lat])
        check(lib().gvm_spmd_run(self.handle, hs, tp, cnt, n, steps, dev, launch, host, lp), "gvm_spmd_run")
        out = (list(dev)[:steps], list(launch)[:steps], list(host)[:steps])
        if latency:
            out += ([[v / 1e9 for v in list(x)[:steps * len(a)]] for x, a in zip(lat, task_arrays)],)
        return out

    def spmd_run_overlapped(self, ranks, arrays_even, arrays_odd, steps: int) -> tuple[float, list[float]]:
        """gvm_spmd_run_overlapped: like spmd_run with two steps in flight per
        rank (step i + 1 submitted before step i is collected); even steps use
        arrays_even, odd steps arrays_odd (None: the same). Returns (total ms,
        per-step ms at which each step's results were all collected)."""
        n = len(ranks)
        hs = (c_void_p * n)(*[r.handle for r in ranks])
        te = (ctypes.POINTER(GvmTask) * n)(*[ctypes.cast(a, ctypes.POINTER(GvmTask)) for a in arrays_even])
        to = None
        if arrays_odd is not None:
            to = (ctypes.POINTER(GvmTask) * n)(*[ctypes.cast(a, ctypes.POINTER(GvmTask)) for a in arrays_odd])
        cnt = (ctypes.c_uint32 * n)(*[len(a) for a in arrays_even])
        total = ctypes.c_double()
        done = (ctypes.c_double * max(steps, 1))()
        check(lib().gvm_spmd_run_overlapped(self.handle, hs, te, to, cnt, n, steps, byref(total), done),
              "gvm_spmd_run_overlapped")
        return total.value, list(done)[:steps]

    def spmd_run_pipelined(self, ranks, arrays_by_phase, steps: int) -> tuple[float, list[float]]:
        """gvm_spmd_run_pipelined: like spmd_run_overlapped with
        len(arrays_by_phase) steps in flight per rank; step i uses
        arrays_by_phase[i % len(arrays_by_phase)] (one list of per-rank ctypes
        task arrays per phase). Returns (total ms, per-step ms at which each
        step's results were all collected)."""
        n = len(ranks)
        P = len(arrays_by_phase)
        hs = (c_void_p * n)(*[r.handle for r in ranks])
        per = [(ctypes.POINTER(GvmTask) * n)(*[ctypes.cast(a, ctypes.POINTER(GvmTask)) for a in arrs])
               for arrs in arrays_by_phase]
        ph = (ctypes.POINTER(ctypes.POINTER(GvmTask)) * P)(
            *[ctypes.cast(x, ctypes.POINTER(ctypes.POINTER(GvmTask))) for x in per])
        cnt = (ctypes.c_uint32 * n)(*[len(a) for a in arrays_by_phase[0]])
        total = ctypes.c_double()
        done = (ctypes.c_double * max(steps, 1))()
        check(lib().gvm_spmd_run_pipelined(self.handle, hs, ph, P, cnt, n, steps, byref(total), done),
              "gvm_spmd_run_pipelined")
        return total.value, list(done)[:steps]

    def open_loop_run(self, ranks, task_arrays, arrival_ns, max_inflight: int = 0):
        """gvm_open_loop_run: rank i submits task_arrays[i][j] (ctypes arrays
        of GvmTask) at arrival_ns[i][j] ns after a common start (one native
        thread per rank). Returns (span seconds, per-rank latency lists in
        seconds: completion seen minus scheduled arrival)."""
        n = len(ranks)
        hs = (c_void_p * n)(*[r.handle for r in ranks])
        tp = (ctypes.POINTER(GvmTask) * n)(*[ctypes.cast(a, ctypes.POINTER(GvmTask)) for a in task_arrays])
        arr = [(ctypes.c_uint64 * max(len(a), 1))(*[int(x) for x in a]) for a in arrival_ns]
        ap = (ctypes.POINTER(ctypes.c_uint64) * n)(*[ctypes.cast(a, ctypes.POINTER(ctypes.c_uint64)) for a in arr])
        cnt = (ctypes.c_uint32 * n)(*[len(a) for a in task_arrays])
        lat = [(ctypes.c_double * max(len(a), 1))() for a in task_arrays]
        lp = (ctypes.POINTER(ctypes.c_double) * n)(*[ctypes.cast(x, ctypes.POINTER(ctypes.c_double)) for x in lat])
        span = ctypes.c_double()
        check(lib().gvm_open_loop_run(self.handle, hs, tp, ap, cnt, n, max_inflight, lp, byref(span)),
              "gvm_open_loop_run")
        return span.value / 1e9, [[v / 1e9 for v in list(l)[: len(a)]] for l, a in zip(lat, task_arrays)]

    def shutdown(self) -> None:
        if getattr(self, "handle", None) is not None:
            rc = lib().gvm_shutdown(self.handle)
            if rc != _abi.GVM_ESTATE:  # an IPC server still serves it: nothing was freed
                self.handle = None
            check(rc, "gvm_shutdown")
            # The device memory goes back to PyTorch's allocator now, not when
            # the last reference to this object goes away.
            self.arena = None
            self.ctrl = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.shutdown()

    def __del__(self):
        # The arena and control block are torch allocations: a manager dropped
        # without shutdown (a resident scheduler still running) must stop
        # before the caching allocator can hand that memory to other tensors.
        try:
            self.shutdown()
        except Exception:
            pass


def vadd_f32(a: torch.Tensor, b: torch.Tensor, c: torch.Tensor, stream=None) -> None:
    """c = a + b on the device (the vector-add task kernel alone)."""
    check(lib().gvm_vadd_f32(_ptr(a), _ptr(b), _ptr(c), a.numel(), _stream_handle(stream)), "gvm_vadd_f32")


def vmul_f32(a: torch.Tensor, b: torch.Tensor, c: torch.Tensor, iters: int, stream=None) -> None:
    """c = a * b * ... * b (`iters` float32 products) on the device (the vector-multiply task kernel alone)."""
    check(
        lib().gvm_vmul_f32(_ptr(a), _ptr(b), _ptr(c), a.numel(), iters, _stream_handle(stream)), "gvm_vmul_f32"
    )


def sgemm_scratch_bytes(m: int, n: int, k: int, path: str = "split3") -> int:
    return lib().gvm_sgemm_scratch_bytes(m, n, k, _PATHS[path])


def sgemm_f32(
    A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, path: str = "split3", scratch: torch.Tensor | None = None,
    stream=None,
) -> None:
    """C = A B on the device (the matrix-multiply task kernel alone)."""
    m, k = A.shape
    n = B.shape[1]
    sp, sb = 0, 0
    if path == "split3":
        need = sgemm_scratch_bytes(m, n, k, path)
        if scratch is None:
            scratch = torch.empty(need + 256, dtype=torch.uint8, device=A.device)
        sp = (scratch.data_ptr() + 255) // 256 * 256
        sb = scratch.numel() - (sp - scratch.data_ptr())
    check(
        lib().gvm_sgemm_f32(_ptr(A), _ptr(B), _ptr(C), m, n, k, _PATHS[path], sp, sb, _stream_handle(stream)),
        "gvm_sgemm_f32",
    )


def kernel_status() -> int:
    v = c_uint32(0)
    check(lib().gvm_kernel_status(byref(v)), "gvm_kernel_status")
    return v.value
