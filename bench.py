#!/usr/bin/env python3
"""Throughput of SPMD ranks sharing one GB300 through the gvm manager.

Workload (default): 16 ranks (one GPU shared by 16 CPU cores), each
submitting 64 SGEMM tasks C = A B with M = N = K = 512, A and B standard
normal from seed rank*1000 + task (B from seed + 2^32). One step is the whole
hot path over that batch: every rank submits its 64 tasks (gvm_submit_many),
the request barrier flushes them (gvm_flush launches the persistent
scheduler), every rank syncs (gvm_sync).

  value  tasks/s with the operands resident in HBM (GVM_TASK_RESIDENT),
         timed with CUDA events on the scheduler stream around each step.
  e2e    tasks/s through the same API with pinned host buffers: the input
         copies, the kernel and the output copies are inside the timed
         region (host wall clock).
  roofline     the scheduler kernel (the dominant kernel: it runs every tile)
         against its compute roof (SGEMM: bf16 / 3 or FFMA), with HBM under
         `other` and the roof with the longer time floor named in `binding`
  cpu_baseline the CPU oracle (binary64) on the host cores, bounded sample
  plain_per_rank  each rank in its own process and context, default stream,
         the same task kernels (Section 4.1's conventional sharing, Eq. 1):
         operands resident, with copies, and with T_init

``--impl reference`` runs the reference arm: the CPU oracle as it stands on
the host cores, one rank per thread, a bounded sample per step.

Multi-GPU (torchrun): each process runs its own replica of the workload on
its GPU (ranks are independent; no collective on the data path), and value
is the tasks of all replicas over the slowest replica's time (weak scaling).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "tasks/s & GB/s, N ranks on 1 GB300, shared vs per-rank; p50/p99 task latency"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
GB300_SMS = 152
FP32_LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["gvm", "reference"], default="gvm")
    p.add_argument("--workload", choices=["sgemm512", "vadd_tiny", "vadd_hbm", "serving", "grouped", "stress"],
                   default="sgemm512")
    p.add_argument("--serving-tasks", type=int, default=0, help="serving workload: total tasks (default 4096)")
    p.add_argument("--repeats", type=int, default=3, help="serving and stress: runs per load point")
    p.add_argument("--duration", type=float, default=10.0,
                   help="stress: seconds of arrivals per load point (the configuration's is 60)")
    p.add_argument("--path", choices=["split3", "split3_wide", "split3_tma", "fma"], default=None,
                   help="SGEMM arithmetic and tile form (default: the autotuner's split3 form)")
    p.add_argument("--mode", choices=["barrier", "continuous"], default="barrier")
    p.add_argument("--skip-e2e", action="store_true")
    p.add_argument("--skip-cpu", action="store_true")
    p.add_argument("--skip-plain", action="store_true", help="skip the plain one-context-per-rank forms")
    p.add_argument("--skip-extra", action="store_true",
                   help="skip the FMA, vector-add and plain-form legs of the default workload")
    p.add_argument("--model", action="store_true", help="also check timings against Eqs. 1, 2 and 7")
    p.add_argument("--e2e-overlap", type=int, choices=[1, 2, 3, 4], default=2,
                   help="end-to-end leg: steps in flight per rank (>= 2: gvm_spmd_run_pipelined, own manager)")
    p.add_argument("--direct-output", type=int, choices=[0, 1], default=None,
                   help="host-mode results written by the scheduler into the host buffers (default: tuning)")
    p.add_argument("--cross-process", action="store_true",
                   help="also run the workload end to end with every rank a separate client process")
    p.add_argument("--ipc-client", nargs=2, metavar=("NAME", "RANK"), help=argparse.SUPPRESS)
    p.add_argument("--paper-modes", action="store_true",
                   help="also run the workload in the paper's host-issued PS-1 / PS-2 modes")
    p.add_argument("--quantum", type=int, default=8)
    p.add_argument("--copy-streams-max", type=int, default=0,
                   help="copy streams the managers create (0: the library's default budget)")
    p.add_argument("--e2e-steps", type=int, default=0,
                   help="timed steps of the end-to-end leg (0: half of --steps)")
    p.add_argument("--copy-in-streams", type=int, default=0,
                   help="input copy streams of the manager (0: half of the copy-stream limit)")
    p.add_argument("--idle-poll-ns", type=int, default=1000,
                   help="sleep of an idle scheduler CTA between polls of the task rings")
    p.add_argument("--vadd-tile", type=int, default=None,
                   help="elements per vector-add tile (0: per task, n / CTAs; default: the tuned value)")
    p.add_argument("--copy-run-mb", type=int, default=None,
                   help="merge adjacent host-mode copies up to this many MiB (default: the tuned choice)")
    p.add_argument("--l2-prefetch", type=int, choices=[0, 1], default=None,
                   help="split3: prefetch the next queued tile's operands into L2 (default: the tuned choice)")
    p.add_argument("--harness", choices=["native", "python"], default="native",
                   help="rank threads: native (gvm_spmd_run) or Python threads calling the API")
    p.add_argument("--ranks", type=int, default=0, help="smaller case for profiling (not a bench line)")
    p.add_argument("--per-rank", type=int, default=0, help="smaller case for profiling (not a bench line)")
    return p.parse_args()


# --------------------------------------------------------------- workloads


def workload(name, ranks=0, per_rank=0):
    if name == "sgemm512":
        R, P = ranks or 16, per_rank or 64
        w = synth.sgemm_square(ranks=R, per_rank=P, side=512)
        desc = f"SGEMM M=N=K=512, {R} ranks x {P} tasks, standard-normal operands"
    elif name == "vadd_hbm":
        R, P = ranks or 16, per_rank or 4
        w = synth.vadd_tiny(ranks=R, per_rank=P, n=1 << 22)
        desc = f"vector add n=2^22, {R} ranks x {P} tasks, uniform [-1,1) operands"
    else:
        R, P = ranks or 4, per_rank or 8
        w = synth.vadd_tiny(ranks=R, per_rank=P, n=65536)
        desc = f"vector add n=65536, {R} ranks x {P} tasks, uniform [-1,1) operands"
    return w, desc


def task_inputs(spec):
    if spec.kind == synth.TASK_VADD:
        return synth.vadd_inputs(spec.seed, spec.n)
    return synth.sgemm_inputs(spec.seed, spec.m, spec.n, spec.k)


_INPUTS = {}


def gen_inputs(w):
    """Every task's operands, generated once per workload and process."""
    key = (w.name, w.ranks, len(w.tasks))
    if key not in _INPUTS:
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            _INPUTS[key] = list(ex.map(task_inputs, w.tasks))
    return _INPUTS[key]


# --------------------------------------------------------------- clocks


class ClockSampler:
    FIELDS = (
        "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.rows = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
            )
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def summary(self):
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower() == "active":
                    reasons.add(nm)
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons),
            "samples": len(self.rows),
        }


# --------------------------------------------------------------- helpers


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return FALLBACK_PEAKS, "fallback"


# The sources the scheduler kernels are compiled from (host code does not
# change their DRAM traffic per tile).
KERNEL_SOURCES = ("gvm_sched.cu", "gvm_fused.cuh", "gvm_wide.cuh", "gvm_tma.cuh", "gvm_device.cuh", "gvm_internal.h")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1511_07658_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(key):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources and the same workload; else None."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
    except OSError:
        return None
    e = t.get(key)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("bytes_per_launch")


def max_over_ranks(x: float, world: int) -> float:
    """The largest value of x over the ranks of the process group (the time
    of the slowest rank); x itself when running alone. NCCL reduces a CUDA
    tensor, gloo a CPU one."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: int, steps: int, world: int, slowest_s: float) -> float:
    """Units all ranks processed per second of the slowest rank (ranks run
    independent replicas of the workload: weak scaling)."""
    return units_per_rank_step * steps * world / slowest_s


def host_memcpy_gbs(nbytes=256 << 20, reps=3):
    """Host memory copy rate (read + write bytes per second) right after a
    host-link-bound leg: context for its number, since other jobs on the
    same host share the memory system the copies go through."""
    a = np.ones(nbytes, dtype=np.uint8)
    b = np.empty_like(a)
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        np.copyto(b, a)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return 2 * nbytes / best / 1e9


def sgemm_roofline(tasks, launch_s, path, pk, pk_kind):
    """Roofline of an SGEMM launch against both of its roofs: the compute
    roof of its path (split3: the measured bf16 burst / 3 products; FMA: the
    FP32 lanes at the maximum clock), reported as the bound, and HBM (A, B
    and C once per task, 4 (mk + kn + mn) bytes) under `other`, with
    `binding` naming the roof whose time floor (work / peak) is longer."""
    flops = sum(s.flops for s in tasks)
    byts = sum(4 * (s.m * s.k + s.k * s.n + s.m * s.n) for s in tasks)
    if path == "fma":
        cpeak = GB300_SMS * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        compute = {"bound": "alu", "unit": "TFLOP/s", "peak_basis": "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"}
    else:
        cpeak = pk["bf16_tflops"] / 3.0
        compute = {"bound": "tensor", "unit": "TFLOP/s",
                   "peak_basis": f"bf16 dense {pk['bf16_tflops']} TFLOP/s ({pk_kind}, burst) / 3 products"}
    compute.update({"achieved": flops / launch_s / 1e12, "peak": cpeak, "algorithmic_flops": flops})
    compute["frac"] = compute["achieved"] / cpeak
    hbm = {"bound": "hbm", "unit": "GB/s", "peak_basis": f"HBM copy {pk['hbm_gbs']} GB/s ({pk_kind})",
           "achieved": byts / launch_s / 1e9, "peak": pk["hbm_gbs"], "bytes_per_launch": byts}
    hbm["frac"] = hbm["achieved"] / hbm["peak"]
    main = dict(compute)
    main["other"] = {k: hbm[k] for k in ("bound", "unit", "achieved", "peak", "frac", "bytes_per_launch")}
    main["binding"] = "hbm" if hbm["frac"] > compute["frac"] else compute["bound"]
    return main


def block_link_gbs(blocks, to_device: bool):
    """Copy rate of each page-locked host block on its own (one copy of the
    whole block, best of 2, CUDA events): in a virtual machine each
    allocation's placement relative to the GPU's host link is not visible,
    so this shows whether a slow end-to-end leg had slow buffers. The blocks'
    contents are left as they were. Returns min, median and max over the
    blocks (GB/s)."""
    import torch

    rates = []
    for hb in blocks:
        # The device copy starts as the block's own bytes, so that timing the
        # device-to-host direction writes back what the block already holds.
        dev = hb.to("cuda")
        best = None
        for _ in range(2):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            if to_device:
                dev.copy_(hb, non_blocking=True)
            else:
                hb.copy_(dev, non_blocking=True)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        rates.append(hb.numel() / (best / 1e3) / 1e9)
        del dev
    rates.sort()
    return {"min": rates[0], "median": rates[len(rates) // 2], "max": rates[-1], "blocks": len(rates)}


def percentile(xs, q):
    if not xs:
        return None
    xs = sorted(xs)
    i = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[i]


# --------------------------------------------------------------- GPU arm


def build_tasks(w, inputs, resident, bufs):
    """Per rank, a ctypes array of GvmTask for one step."""
    import paper_1511_07658_gb300 as g

    by_rank = [[] for _ in range(w.ranks)]
    for spec, inp in zip(w.tasks, inputs):
        by_rank[spec.rank].append((spec, inp))
    arrays = []
    for r, lst in enumerate(by_rank):
        arr = (g.GvmTask * len(lst))()
        for i, (spec, inp) in enumerate(lst):
            t = arr[i]
            t.type = g.GVM_TASK_VADD if spec.kind == synth.TASK_VADD else g.GVM_TASK_SGEMM
            t.n = spec.n
            t.m, t.k = spec.m, spec.k
            if resident:
                t.flags = g.GVM_TASK_RESIDENT
                t.a_off, t.b_off, t.c_off = bufs["res_offs"][(r, spec.index)]
            else:
                t.flags = 0
                a, b, c = bufs["host"][(r, spec.index)]
                t.a, t.b, t.c = a.data_ptr(), b.data_ptr(), c.data_ptr()
        arrays.append(arr)
    return arrays


def run_step(mgr, ranks, arrays, pool, record=True):
    """Every rank submits its batch (one thread per rank), flush, sync all.
    With ``record``, CUDA events on the scheduler stream bracket the flush's
    launch (barrier mode only: a resident scheduler never completes)."""
    def submit(r):
        first, cnt = ranks[r].submit_many(arrays[r])
        return first + cnt - 1

    h0 = time.perf_counter()
    lasts = list(pool.map(submit, range(len(ranks))))
    h1 = time.perf_counter()
    ev0 = ev1 = None
    import torch

    if record:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(mgr.sched_stream)
    mgr.flush()
    if record:
        ev1.record(mgr.sched_stream)
    h2 = time.perf_counter()
    list(pool.map(lambda r: ranks[r].sync(lasts[r]), range(len(ranks))))
    h3 = time.perf_counter()
    HOST_TIMES.append((h1 - h0, h2 - h1, h3 - h2))
    return ev0, ev1, lasts


HOST_TIMES = []  # per step: (submit, flush, sync) host seconds


def paper_modes_check(args, g, w, slice_bytes, resident, res_arrays, host_arrays, host, res_offs, tasks_per_step):
    """The same workload through the same API in the paper's own mechanism
    (GVM_MODE_PS1 / GVM_MODE_PS2: the manager's host thread issues every
    task's copies and kernel on its rank's stream at the request barrier;
    Sections 4.2.1 and 5) instead of the persistent scheduler: tasks/s with
    device-resident operands (host clock around each native SPMD step) and
    end to end from the same pinned host buffers."""
    R = w.ranks
    per_rank = len(w.tasks) // R
    out = {}
    for mode in ("ps1", "ps2"):
        mgr = g.Manager(R, ring_depth=max(2, 1 << (per_rank - 1).bit_length()), mode=mode, sgemm_path=args.path,
                        slice_bytes=slice_bytes, resident_bytes=resident)
        ranks = [mgr.attach(r) for r in range(R)]
        for spec in w.tasks:
            ta, tb, _ = host[(spec.rank, spec.index)]
            oa, ob, _ = res_offs[(spec.rank, spec.index)]
            ranks[spec.rank].write(oa, ta)
            ranks[spec.rank].write(ob, tb)
        row = {}
        for leg, arrays in (("value", res_arrays), ("e2e", host_arrays)):
            mgr.spmd_run(ranks, arrays, max(1, args.warmup))
            steps = args.steps if leg == "value" else max(3, args.steps // 2)
            _, _, hst = mgr.spmd_run(ranks, arrays, steps)
            row[leg] = tasks_per_step * steps / (sum(hst) / 1e3)
        row["kernel_launches_per_step"] = tasks_per_step
        out[mode] = row
        mgr.shutdown()
    return out


def _ipc_layout(w):
    """Per rank: byte offsets (a, b, c) of each task in the rank's data area
    (256-byte aligned, inputs and output of a task adjacent) and the total."""
    offs, need = {}, [0] * w.ranks
    for spec in w.tasks:
        if spec.kind in (synth.TASK_VADD, synth.TASK_VMUL):
            la = lb = lc = 4 * spec.n
        else:
            la, lb, lc = 4 * spec.m * spec.k, 4 * spec.k * spec.n, 4 * spec.m * spec.n
        o = need[spec.rank]
        a256 = lambda x: (x + 255) // 256 * 256  # noqa: E731
        offs[(spec.rank, spec.index)] = (o, o + a256(la), o + a256(la) + a256(lb))
        need[spec.rank] = o + a256(la) + a256(lb) + a256(lc)
    return offs, need


def ipc_client_main(args):
    """One client process of the cross-process leg (no CUDA): fills its data
    area with its tasks' inputs, then runs warm-up and timed steps (submit
    every task, arrive at the request barrier, wait for every result) and
    prints its timed seconds."""
    from paper_1511_07658_gb300 import GVM_EAGAIN, GvmError
    from paper_1511_07658_gb300.ipc import IpcClient

    name, rank = args.ipc_client[0], int(args.ipc_client[1])
    w, _ = workload(args.workload, args.ranks, args.per_rank)
    offs, _ = _ipc_layout(w)
    mine = [s for s in w.tasks if s.rank == rank]
    c = IpcClient(name, rank)
    for spec in mine:
        a, b = task_inputs(spec)
        oa, ob, _ = offs[(rank, spec.index)]
        c.floats(oa, a.size)[:] = np.ascontiguousarray(a).ravel()
        c.floats(ob, b.size)[:] = np.ascontiguousarray(b).ravel()

    def step():
        seqs = []
        for spec in mine:
            oa, ob, oc = offs[(rank, spec.index)]
            while True:
                try:
                    if spec.kind == synth.TASK_SGEMM:
                        seqs.append(c.submit_sgemm(oa, ob, oc, spec.m, spec.n, spec.k))
                    else:
                        seqs.append(c.submit_vadd(oa, ob, oc, spec.n))
                    break
                except GvmError as e:  # ring full: let the barrier drain it
                    if e.code != GVM_EAGAIN:
                        raise
                    c.barrier()
                    c.wait(seqs[-1], timeout_s=60)
        c.barrier()
        for q in seqs:
            c.wait(q, timeout_s=60)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    c.close()
    print(json.dumps({"rank": rank, "seconds": dt}))


def cross_process_check(args, w):
    """The workload end to end with every rank a separate client process
    (include/gvm_ipc.h): operands and results in each rank's shared-memory
    data area, copies between it and the GPU inside the timed region, the
    request barrier across processes. tasks/s = all ranks' tasks of the timed
    steps / the slowest client's timed seconds."""
    import subprocess

    import paper_1511_07658_gb300 as g

    R = w.ranks
    per_rank = len(w.tasks) // R
    _, need = _ipc_layout(w)
    name = f"gvmbench-{os.getpid()}"
    region = g.IpcRegion.create(name, R, max(need), max(2, 1 << (per_rank - 1).bit_length()))
    try:
        with g.Manager(R, ring_depth=max(2, 1 << (per_rank - 1).bit_length()), mode="barrier",
                       sgemm_path=args.path, slice_bytes=max(need) + (64 << 20)) as mgr:
            server = g.IpcServer(mgr, region)
            try:
                cmd = [sys.executable, os.path.abspath(__file__), "--workload", args.workload, "--steps",
                       str(max(3, args.steps // 2)), "--warmup", str(max(1, args.warmup))]
                if args.ranks:
                    cmd += ["--ranks", str(args.ranks), "--per-rank", str(args.per_rank)]
                procs = [subprocess.Popen(cmd + ["--ipc-client", name, str(r)], stdout=subprocess.PIPE,
                                          stderr=subprocess.PIPE, text=True) for r in range(R)]
                outs = [p.communicate(timeout=600) for p in procs]
                counts = server.counts()
            finally:
                server.stop()
    finally:
        region.destroy()
    secs = []
    for p, (o, e) in zip(procs, outs):
        if p.returncode != 0:
            raise RuntimeError(f"ipc client failed: {e[-2000:]}")
        secs.append(json.loads(o.strip().splitlines()[-1])["seconds"])
    steps = max(3, args.steps // 2)
    return {"value": R * per_rank * steps / max(secs), "unit": "tasks/s", "clients": R, "steps": steps,
            "kind": "end to end, one process per rank, data in POSIX shared memory",
            "barriers": counts["barriers"], "tasks_completed": counts["completed"]}


def gpu_arm(args, w, desc, rank, world):
    import torch

    import paper_1511_07658_gb300 as g

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    inputs = gen_inputs(w)
    R = w.ranks
    per_rank = len(w.tasks) // R
    # resident region: every task's operands and result
    sizes = {}
    res_offs = {}
    res_need = [0] * R
    for spec in w.tasks:
        if spec.kind == synth.TASK_VADD:
            la = lb = lc = 4 * spec.n
        else:
            la, lb, lc = 4 * spec.m * spec.k, 4 * spec.k * spec.n, 4 * spec.m * spec.n
        off = res_need[spec.rank]
        res_offs[(spec.rank, spec.index)] = (off, off + la, off + la + lb)
        res_need[spec.rank] = off + (la + lb + lc + 255) // 256 * 256
        sizes[(spec.rank, spec.index)] = (la, lb, lc)
    resident = max(res_need)
    # Several steps in flight on the end-to-end leg (its own manager, whose
    # ring and staging hold that many batches).
    overlap = args.e2e_overlap if (args.harness == "native" and args.mode != "continuous") else 1
    host_stage = max(sum(sizes[(s.rank, s.index)]) for s in w.tasks) * per_rank
    slice_bytes = resident + host_stage + (64 << 20)
    slice_bytes = (slice_bytes + (1 << 20) - 1) // (1 << 20) * (1 << 20)
    mgr = g.Manager(
        R, ring_depth=max(2, 1 << (per_rank - 1).bit_length()), mode=args.mode, sgemm_path=args.path,
        slice_bytes=slice_bytes, resident_bytes=resident, ingest_quantum=args.quantum,
        direct_output=None if args.direct_output is None else bool(args.direct_output),
        l2_prefetch=None if args.l2_prefetch is None else bool(args.l2_prefetch),
        copy_run_bytes=None if args.copy_run_mb is None else args.copy_run_mb << 20,
        copy_streams_max=args.copy_streams_max, vadd_tile=args.vadd_tile,
        idle_poll_ns=args.idle_poll_ns, copy_in_streams=args.copy_in_streams,
    )
    direct_output_used = mgr.cfg.direct_output
    ranks = [mgr.attach(r) for r in range(R)]
    # Host buffers: per rank, one pinned block holding every task's A then B
    # in submission order and one holding the outputs, each operand at a
    # 256-byte multiple (as a rank of an SPMD program would keep its batch);
    # the manager merges copies that are adjacent on both sides.
    def al256(x):
        return (x + 255) // 256 * 256

    in_off, out_off = {}, {}
    in_need, out_need = [0] * R, [0] * R
    for spec in w.tasks:
        la, lb, lc = sizes[(spec.rank, spec.index)]
        in_off[(spec.rank, spec.index)] = in_need[spec.rank]
        in_need[spec.rank] += al256(la) + al256(lb)
        out_off[(spec.rank, spec.index)] = out_need[spec.rank]
        out_need[spec.rank] += al256(lc)
    in_blocks = [torch.empty(max(n, 256), dtype=torch.uint8).pin_memory() for n in in_need]
    out_blocks = [torch.empty(max(n, 256), dtype=torch.uint8).pin_memory() for n in out_need]
    # steps of the pipelined end-to-end leg write to the output blocks of
    # their phase (step i: phase i % overlap), so that a step's results stay
    # until its rank has collected them
    out_blocks_ph = [out_blocks] + [[torch.empty(max(n, 256), dtype=torch.uint8).pin_memory() for n in out_need]
                                    for _ in range(overlap - 1)]

    def view(block, off, nbytes):
        return block[off:off + nbytes].view(torch.float32)

    host = {}
    host_ph = [host] + [{} for _ in range(overlap - 1)]
    for spec, inp in zip(w.tasks, inputs):
        a, b = inp
        la, lb, lc = sizes[(spec.rank, spec.index)]
        io = in_off[(spec.rank, spec.index)]
        ta = view(in_blocks[spec.rank], io, la)
        tb = view(in_blocks[spec.rank], io + al256(la), lb)
        ta.copy_(torch.from_numpy(np.ascontiguousarray(a)).reshape(-1))
        tb.copy_(torch.from_numpy(np.ascontiguousarray(b)).reshape(-1))
        tc = view(out_blocks[spec.rank], out_off[(spec.rank, spec.index)], lc)
        host[(spec.rank, spec.index)] = (ta, tb, tc)
        for ph in range(1, overlap):
            host_ph[ph][(spec.rank, spec.index)] = (
                ta, tb, view(out_blocks_ph[ph][spec.rank], out_off[(spec.rank, spec.index)], lc))
        oa, ob, _ = res_offs[(spec.rank, spec.index)]
        ranks[spec.rank].write(oa, ta)
        ranks[spec.rank].write(ob, tb)
    bufs = {"res_offs": res_offs, "host": host}
    res_arrays = build_tasks(w, inputs, True, bufs)
    host_arrays = build_tasks(w, inputs, False, bufs)
    host_arrays_ph = [host_arrays] + [build_tasks(w, inputs, False, {"res_offs": res_offs, "host": host_ph[ph]})
                                      for ph in range(1, overlap)]
    pool = ThreadPoolExecutor(max_workers=R)
    sampler = ClockSampler(dev)

    # ---- device-resident value
    cont = args.mode == "continuous"

    def device_sync():
        # A resident (continuous-mode) scheduler never finishes before
        # shutdown, so only barrier mode may synchronise the whole device.
        if not cont:
            torch.cuda.synchronize()

    native = args.harness == "native"

    host_lat = []  # host-clock latency of every timed task (s), when the harness records it

    def native_steps(arrays, steps, latency=False):
        # One native thread per rank (gvm_spmd_run). The resident scheduler of
        # continuous mode holds the scheduler stream, so no events there.
        if cont:
            n = len(ranks)
            hs = (ctypes.c_void_p * n)(*[r.handle for r in ranks])
            tp = (ctypes.POINTER(g.GvmTask) * n)(*[ctypes.cast(a, ctypes.POINTER(g.GvmTask)) for a in arrays])
            cnt = (ctypes.c_uint32 * n)(*[len(a) for a in arrays])
            host = (ctypes.c_double * max(steps, 1))()
            rc = g._abi.lib().gvm_spmd_run(mgr.handle, hs, tp, cnt, n, steps, None, None, host, None)
            g._abi.check(rc, "gvm_spmd_run")
            return [h / 1e3 for h in list(host)[:steps]], [h / 1e3 for h in list(host)[:steps]]
        if latency:
            dev, launch, _, lat = mgr.spmd_run(ranks, arrays, steps, latency=True)
            for x in lat:
                host_lat.extend(x)
        else:
            dev, launch, _ = mgr.spmd_run(ranks, arrays, steps)
        return [d / 1e3 for d in dev], [x / 1e3 for x in launch]

    if native:
        native_steps(res_arrays, args.warmup)
    else:
        for _ in range(args.warmup):
            run_step(mgr, ranks, res_arrays, pool, record=not cont)
    device_sync()
    if world > 1:
        torch.distributed.barrier()
    sampler.start()
    t_step = []
    t_kernel = []
    wall0 = time.perf_counter()
    if native:
        if not cont:
            st0 = torch.cuda.Event(enable_timing=True)
            st1 = torch.cuda.Event(enable_timing=True)
            st0.record(mgr.sched_stream)
        t_step, t_kernel = native_steps(res_arrays, args.steps)
        # Sequence numbers are per rank, from 0: warm-up steps, then timed ones.
        lasts = [(args.warmup + args.steps) * len(res_arrays[r]) - 1 for r in range(R)]
        if not cont:
            st1.record(mgr.sched_stream)
            torch.cuda.synchronize()
            total_s = st0.elapsed_time(st1) / 1e3
        else:
            total_s = time.perf_counter() - wall0
        wall = time.perf_counter() - wall0
    elif not cont:
        st0 = torch.cuda.Event(enable_timing=True)
        st1 = torch.cuda.Event(enable_timing=True)
        st0.record(mgr.sched_stream)
        events = []
        for _ in range(args.steps):
            e_step0 = torch.cuda.Event(enable_timing=True)
            e_step0.record(mgr.sched_stream)
            ev0, ev1, lasts = run_step(mgr, ranks, res_arrays, pool)
            e_step1 = torch.cuda.Event(enable_timing=True)
            e_step1.record(mgr.sched_stream)
            events.append((e_step0, ev0, ev1, e_step1))
        st1.record(mgr.sched_stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        for e_step0, ev0, ev1, e_step1 in events:
            t_step.append(e_step0.elapsed_time(e_step1) / 1e3)
            t_kernel.append(ev0.elapsed_time(ev1) / 1e3)
        total_s = st0.elapsed_time(st1) / 1e3
    else:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            _, _, lasts = run_step(mgr, ranks, res_arrays, pool, record=False)
            t_step.append(time.perf_counter() - t0)
        wall = time.perf_counter() - wall0
        t_kernel = t_step
        total_s = wall
    sampler.stop()
    # device-side service latency of the last step's tasks
    lat = []
    for r, rk in enumerate(ranks):
        for s in range(lasts[r] - per_rank + 1, lasts[r] + 1):
            t0, t1 = rk.task_times(s)
            lat.append((t1 - t0) / 1e3)
    # Host-clock latency (the rank's submit call -> the completion it sees)
    # over a few more steps in which every rank collects its tasks one by one
    # (collecting them one by one adds host time between steps, so these
    # steps are not part of the timed ones).
    lat_steps = min(5, args.steps)
    if native and not cont:
        native_steps(res_arrays, lat_steps, latency=True)
    tasks_per_step = len(w.tasks)
    if world > 1:
        total_s = max_over_ranks(total_s, world)
    value = whole_job_rate(tasks_per_step, args.steps, world, total_s)
    stats_after_value = mgr.stats()
    st = stats_after_value
    ph = st["launch_phase"]
    timeline = {
        "start_to_last_done_us": (st["launch_last_done_ns"] - st["launch_start_ns"]) / 1e3,
        "last_done_to_exit_us": (st["launch_exit_ns"] - st["launch_last_done_ns"]) / 1e3,
        "cta_ms": {"acquire": ph[0] / 1e6, "ingest": ph[1] / 1e6, "stage_wait": ph[2] / 1e6, "gemm": ph[3] / 1e6,
                   "mma_wait": ph[4] / 1e6, "vadd": ph[5] / 1e6, "epilogue": ph[8] / 1e6},
        "tiles": ph[6],
        "ingest_passes": ph[7],
    }
    if HOST_TIMES:
        last = HOST_TIMES[-args.steps:]
        timeline["host_ms_per_step"] = {
            "submit": 1e3 * statistics.mean(h[0] for h in last),
            "flush": 1e3 * statistics.mean(h[1] for h in last),
            "sync": 1e3 * statistics.mean(h[2] for h in last),
        }

    # ---- end to end (host buffers, copies inside the timed region)
    e2e = None
    if not args.skip_e2e and overlap >= 2:
        # `overlap` steps in flight per rank: step i + overlap - 1 is
        # submitted (and flushed) before step i's results are collected; the
        # phases write to separate host output blocks.
        mgr2 = g.Manager(
            R, ring_depth=max(2, 1 << (overlap * per_rank - 1).bit_length()), mode=args.mode, sgemm_path=args.path,
            slice_bytes=overlap * host_stage + (64 << 20), ingest_quantum=args.quantum,
            direct_output=None if args.direct_output is None else bool(args.direct_output),
            l2_prefetch=None if args.l2_prefetch is None else bool(args.l2_prefetch),
            copy_run_bytes=None if args.copy_run_mb is None else args.copy_run_mb << 20,
            copy_streams_max=args.copy_streams_max, vadd_tile=args.vadd_tile,
        idle_poll_ns=args.idle_poll_ns, copy_in_streams=args.copy_in_streams,
        )
        ranks2 = [mgr2.attach(r) for r in range(R)]
        mgr2.spmd_run_pipelined(ranks2, host_arrays_ph, max(1, args.warmup))
        device_sync()
        if world > 1:
            torch.distributed.barrier()
        e_steps = max(3, args.e2e_steps or args.steps // 2)
        total_ms, done_ms = mgr2.spmd_run_pipelined(ranks2, host_arrays_ph, e_steps)
        mgr2.shutdown()
        # per step: time between consecutive steps' results all collected
        gaps_in_order = [b - a for a, b in zip([0.0] + done_ms[:-1], done_ms)]
        gaps = sorted(gaps_in_order)
        h_s = total_ms / 1e3
        if world > 1:
            h_s = max_over_ranks(h_s, world)
        h2d = sum(sizes[k][0] + sizes[k][1] for k in sizes)
        d2h = sum(sizes[k][2] for k in sizes)
        e2e = {
            "value": whole_job_rate(tasks_per_step, e_steps, world, h_s),
            "unit": "tasks/s",
            "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h,
            "host_link_gbs": (h2d + d2h) * e_steps / h_s / 1e9,
            "ms_per_step": 1e3 * h_s / e_steps,
            "steps_in_flight": overlap,
            "host_memcpy_gbs": host_memcpy_gbs(),
            "block_h2d_gbs": block_link_gbs(in_blocks, True),
            "block_d2h_gbs": block_link_gbs(out_blocks, False),
            "step_ms": {"min": gaps[0], "median": gaps[len(gaps) // 2], "max": gaps[-1], "first": gaps_in_order[0],
                        "kind": "host clock, between consecutive steps' results collected (the first from the start)"},
        }
    elif not args.skip_e2e:
        if native:
            native_steps(host_arrays, max(1, args.warmup))
        else:
            for _ in range(max(1, args.warmup)):
                run_step(mgr, ranks, host_arrays, pool, record=not cont)
        device_sync()
        if world > 1:
            torch.distributed.barrier()
        e_steps = max(3, args.steps // 2)
        h0 = time.perf_counter()
        if native:
            native_steps(host_arrays, e_steps)
        else:
            for _ in range(e_steps):
                run_step(mgr, ranks, host_arrays, pool, record=not cont)
        h_s = time.perf_counter() - h0
        if world > 1:
            h_s = max_over_ranks(h_s, world)
        h2d = sum(sizes[k][0] + sizes[k][1] for k in sizes)
        d2h = sum(sizes[k][2] for k in sizes)
        e2e = {
            "value": whole_job_rate(tasks_per_step, e_steps, world, h_s),
            "unit": "tasks/s",
            "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h,
            "host_link_gbs": (h2d + d2h) * e_steps / h_s / 1e9,
            "ms_per_step": 1e3 * h_s / e_steps,
            "host_memcpy_gbs": host_memcpy_gbs(),
            "block_h2d_gbs": block_link_gbs(in_blocks, True),
            "block_d2h_gbs": block_link_gbs(out_blocks, False),
        }

    # ---- parity spot check of the last step (resident outputs), sampled rows
    import oracle

    spot = []
    if e2e is not None and w.tasks[0].kind == synth.TASK_SGEMM:
        # end-to-end outputs (every phase's when several steps were in flight)
        spec = [s for s in w.tasks if s.rank == R - 1][-1]
        inp = inputs[w.tasks.index(spec)]
        rows = np.arange(0, spec.m, 37)
        ref = oracle.sgemm64(inp[0][rows], inp[1])
        for hb in host_ph:
            C = hb[(R - 1, spec.index)][2].reshape(spec.m, spec.n).numpy()
            spot.append(oracle.rel_fro_err(C[rows], ref))
    for r in (0, R - 1):
        spec = [s for s in w.tasks if s.rank == r][-1]
        inp = inputs[w.tasks.index(spec)]
        _, _, oc = res_offs[(r, spec.index)]
        if spec.kind == synth.TASK_SGEMM:
            C = torch.empty(spec.m, spec.n)
            ranks[r].read(oc, C)
            rows = np.arange(0, spec.m, 37)
            err = oracle.rel_fro_err(C.numpy()[rows], oracle.sgemm64(inp[0][rows], inp[1]))
            spot.append(err)
        else:
            c = torch.empty(spec.n)
            ranks[r].read(oc, c)
            spot.append(0.0 if np.array_equal(c.numpy().view(np.uint32), oracle.vadd(*inp).view(np.uint32)) else 1.0)

    mgr.shutdown()
    pool.shutdown()
    paper_modes = None
    if args.paper_modes and not cont:
        paper_modes = paper_modes_check(args, g, w, slice_bytes, resident, res_arrays, host_arrays, host, res_offs,
                                        tasks_per_step)
    pk, pk_kind = peaks()
    kmean = statistics.mean(t_kernel)
    if w.tasks[0].kind == synth.TASK_SGEMM:
        roof = sgemm_roofline(w.tasks, kmean, args.path, pk, pk_kind)
        achieved, peak = roof["achieved"], roof["peak"]
    else:
        byts = sum(12 * s.n for s in w.tasks)
        peak = pk["hbm_gbs"]
        roof = {"bound": "hbm", "unit": "GB/s", "peak_basis": f"HBM copy {pk['hbm_gbs']} GB/s ({pk_kind})"}
        achieved = byts / kmean / 1e9
    kname = {"split3": "sched_fused_kernel", "split3_wide": "sched_wide_kernel",
             "split3_tma": "sched_tma_kernel"}.get(args.path, "sched_fma_kernel")
    key = f"{kname}/{args.workload}"
    roof.update({"kernel": f"gvm::{kname}", "achieved": achieved, "peak": peak,
                 "frac": achieved / peak, "traffic": ncu_traffic(key), "launch_ms": kmean * 1e3})
    clocks = sampler.summary()
    cfg = {
        "workload": desc,
        "ranks": R,
        "tasks_per_rank": per_rank,
        "sgemm_path": args.path,
        "mode": args.mode,
        "direct_output": bool(direct_output_used),
        "l2_prefetch": bool(mgr.cfg.l2_prefetch),
        "copy_run_bytes": int(mgr.cfg.copy_run_bytes),
        "operands": "resident in HBM for value; pinned host buffers for e2e",
        "l2": {"sgemm512": "inputs larger than L2 (2 GiB of operands per step)",
               "vadd_hbm": "inputs larger than L2 (2 GiB of operands per step)"}.get(
                   args.workload, "inputs smaller than L2; latency-bound"),
        "parallelism": f"replicas x{world}" if world > 1 else f"1 GPU, {R} SPMD ranks as host threads",
        "rank_threads": "native (gvm_spmd_run)" if args.harness == "native" else "Python threads",
    }
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "tasks/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16x3->f32" if args.path != "fma" else "f32",
        "data": "synthetic",
        "config": cfg,
        "gbps": {"hbm_operands": sum(sum(v) for v in sizes.values()) * args.steps * world / total_s / 1e9},
        "latency_us": ({"p50": 1e6 * percentile(host_lat, 50), "p99": 1e6 * percentile(host_lat, 99),
                        "p999": 1e6 * percentile(host_lat, 99.9), "tasks": len(host_lat),
                        "kind": f"host clock, the rank's submit call -> completion seen by the rank "
                                f"(gvm_sync per task), every task of {lat_steps} steps after the timed ones"}
                       if host_lat else None),
        "device_latency_us": {"p50": percentile(lat, 50), "p99": percentile(lat, 99),
                              "kind": "device ingest->done, last step"},
        "wall_tasks_per_s": tasks_per_step * args.steps / wall,
        "roofline": roof,
        "sched_timeline_last_launch": timeline,
        "step_ms_distribution": {
            "step": {"min": 1e3 * min(t_step), "median": 1e3 * statistics.median(t_step), "max": 1e3 * max(t_step)},
            "launch": {"min": 1e3 * min(t_kernel), "median": 1e3 * statistics.median(t_kernel),
                       "max": 1e3 * max(t_kernel)},
            "kind": "CUDA events on the scheduler stream per timed step (step: submit to sync; launch: the flush)"},
        "e2e": e2e,
        "gpu_launches": args.steps if not cont else 1,
        "clocks": clocks,
        "parity_spot_rel_err": max(spot) if spot else None,
        "manager_stats": {k: stats_after_value[k] for k in ("launches", "staged_peak", "device_status")},
    }
    if paper_modes is not None:
        out["paper_modes"] = paper_modes
    return out


def resident_leg(args, w, inputs, path, steps, warmup, label):
    """A device-resident leg of its own: a manager on ``path``, every task's
    operands written into its rank's resident region, ``warmup`` then
    ``steps`` SPMD steps (gvm_spmd_run), CUDA events around each scheduler
    launch. Returns tasks/s, the mean launch time, the roofline of the launch
    against the path's bound and a parity spot check of the first and last
    task (vector adds bit-exact in full, SGEMM sampled rows against the
    binary64 oracle)."""
    import torch

    import oracle
    import paper_1511_07658_gb300 as g

    R = w.ranks
    per_rank = len(w.tasks) // R
    res_offs, need, sizes = {}, [0] * R, {}
    for spec in w.tasks:
        if spec.kind == synth.TASK_VADD:
            la = lb = lc = 4 * spec.n
        else:
            la, lb, lc = 4 * spec.m * spec.k, 4 * spec.k * spec.n, 4 * spec.m * spec.n
        off = need[spec.rank]
        res_offs[(spec.rank, spec.index)] = (off, off + la, off + la + lb)
        need[spec.rank] = off + (la + lb + lc + 255) // 256 * 256
        sizes[(spec.rank, spec.index)] = (la, lb, lc)
    resident = max(need)
    slice_bytes = (resident + (64 << 20) + (1 << 20) - 1) // (1 << 20) * (1 << 20)
    mgr = g.Manager(R, ring_depth=max(2, 1 << (per_rank - 1).bit_length()), sgemm_path=path,
                    slice_bytes=slice_bytes, resident_bytes=resident, ingest_quantum=args.quantum)
    try:
        ranks = [mgr.attach(r) for r in range(R)]
        for spec, (a, b) in zip(w.tasks, inputs):
            oa, ob, _ = res_offs[(spec.rank, spec.index)]
            ranks[spec.rank].write(oa, torch.from_numpy(np.ascontiguousarray(a)).reshape(-1))
            ranks[spec.rank].write(ob, torch.from_numpy(np.ascontiguousarray(b)).reshape(-1))
        arrays = build_tasks(w, inputs, True, {"res_offs": res_offs})
        mgr.spmd_run(ranks, arrays, warmup)
        torch.cuda.synchronize()
        dev, launch, _ = mgr.spmd_run(ranks, arrays, steps)
        torch.cuda.synchronize()
        spot = []
        for spec in (w.tasks[0], w.tasks[-1]):
            inp = inputs[w.tasks.index(spec)]
            _, _, oc = res_offs[(spec.rank, spec.index)]
            if spec.kind == synth.TASK_SGEMM:
                C = torch.empty(spec.m, spec.n)
                ranks[spec.rank].read(oc, C)
                rows = np.arange(0, spec.m, 37)
                spot.append(oracle.rel_fro_err(C.numpy()[rows], oracle.sgemm64(inp[0][rows], inp[1])))
            else:
                c = torch.empty(spec.n)
                ranks[spec.rank].read(oc, c)
                same = np.array_equal(c.numpy().view(np.uint32), oracle.vadd(*inp).view(np.uint32))
                spot.append(0.0 if same else 1.0)
        stats = mgr.stats()
    finally:
        mgr.shutdown()
    total_s = sum(dev) / 1e3
    kmean = statistics.mean(launch) / 1e3
    pk, pk_kind = peaks()
    if w.tasks[0].kind == synth.TASK_SGEMM:
        roof = sgemm_roofline(w.tasks, kmean, path, pk, pk_kind)
        achieved, peak = roof["achieved"], roof["peak"]
    else:
        byts = sum(12 * s.n for s in w.tasks)
        peak = pk["hbm_gbs"]
        roof = {"bound": "hbm", "unit": "GB/s", "peak_basis": f"HBM copy {pk['hbm_gbs']} GB/s ({pk_kind})",
                "bytes_per_launch": byts}
        achieved = byts / kmean / 1e9
    kname = {"fma": "sched_fma_kernel", "split3_wide": "sched_wide_kernel",
             "split3_tma": "sched_tma_kernel"}.get(path, "sched_fused_kernel")
    roof.update({"kernel": f"gvm::{kname}", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                 "traffic": ncu_traffic(f"{kname}/{label}"), "launch_ms": kmean * 1e3})
    return {
        "workload": label,
        "value": len(w.tasks) * steps / total_s,
        "unit": "tasks/s",
        "steps": steps,
        "warmup": warmup,
        "ms_per_step": 1e3 * total_s / steps,
        "sgemm_path": path,
        "roofline": roof,
        "parity_spot_rel_err": max(spot),
        "device_status": stats["device_status"],
    }


# --------------------------------------------------------------- CPU oracle


def oracle_rate(w, inputs_fn, max_tasks, threads, min_seconds=0.0):
    """The CPU oracle as it stands: one rank per thread, each rank's first
    tasks in order, until max_tasks tasks are done; the same tasks are run
    again, whole rounds at a time, until at least min_seconds have passed."""
    import oracle

    by_rank = w.by_rank()
    picks = []
    i = 0
    while len(picks) < max_tasks:
        for lst in by_rank:
            if i < len(lst) and len(picks) < max_tasks:
                picks.append(lst[i])
        i += 1
    data = [inputs_fn(s) for s in picks]
    oracle.build()

    def one(j):
        s = picks[j]
        if s.kind == synth.TASK_VADD:
            oracle.vadd(*data[j])
        else:
            oracle.sgemm64(*data[j])

    done = 0
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        while True:
            list(ex.map(one, range(len(picks))))
            done += len(picks)
            if time.perf_counter() - t0 >= min_seconds:
                break
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def cpu_baseline(w):
    threads = min(16, os.cpu_count() or 1)
    n = 2 * threads if w.tasks[0].kind == synth.TASK_SGEMM else len(w.tasks)
    rate, cnt, dt = oracle_rate(w, task_inputs, n, threads, min_seconds=10.0)
    return {"value": rate, "unit": "tasks/s", "cores": threads, "kind": "oracle",
            "sample": f"{cnt} task runs ({n} distinct tasks of the workload, repeated) in {dt:.1f} s, "
                      f"one rank per thread, binary64 SGEMM"}


def reference_arm(args, w, desc):
    threads = min(16, os.cpu_count() or 1)
    n = threads if w.tasks[0].kind == synth.TASK_SGEMM else len(w.tasks)
    for _ in range(args.warmup):
        oracle_rate(w, task_inputs, n, threads)
    total = 0.0
    cnt_all = 0
    for _ in range(args.steps):
        rate, cnt, dt = oracle_rate(w, task_inputs, n, threads)
        total += dt
        cnt_all += cnt
    value = cnt_all / total
    sample = f"{n} tasks per step (one per rank thread) of the workload, binary64 SGEMM"
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "tasks/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": desc, "ranks": w.ranks, "tasks_per_rank": len(w.tasks) // w.ranks},
        "cpu_baseline": {"value": value, "unit": "tasks/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "tasks/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# --------------------------------------------------------------- plain form


def plain_per_rank(w, inputs, phases, init="before", timeout_s=300.0):
    """The plain, non-virtualized form (Section 4.1, Eq. 1): each rank is a
    process of its own (``gvm_plain_rank``, a C client of the library) with
    its own CUDA context on the default stream, running its tasks one after
    another through the same standalone task kernel. Each process is pinned
    to its own core, as the paper pins its processes. ``phases`` is a list of
    (path, mode): path "fma" or "split3" (the fused split3 kernel), mode
    "resident" (operands on the device before the start, kernel +
    synchronize per task) or "copy" (synchronous copies of A, B in and C out
    around every kernel). ``init`` "before": context creation, device
    allocation and page-locking happen before the first start; "timed":
    inside the first phase's timed region (T_init of Eq. 1).

    Every process is started and told to go at once, phase after phase; a
    phase's turnaround is from the first process's start to the last one's
    end (CLOCK_MONOTONIC, shared by the processes). Each phase's last task of
    the first and last rank is checked against the oracle on sampled rows."""
    import select
    import shutil
    import tempfile

    import oracle
    from paper_1511_07658_gb300 import build as gb

    exe = gb.build_plain()
    R = w.ranks
    specs = [[] for _ in range(R)]
    for spec, inp in zip(w.tasks, inputs):
        specs[spec.rank].append((spec, inp))
    per_rank = len(specs[0])
    m, n, k = specs[0][0][0].m, specs[0][0][0].n, specs[0][0][0].k
    path_no = {"fma": 0, "split3": 2}
    tmp = tempfile.mkdtemp(prefix="gvm_plain_", dir="/dev/shm" if os.path.isdir("/dev/shm") else None)
    cores = sorted(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else []
    procs = []
    deadline = time.time() + timeout_s

    def readline(p):
        # one line of a rank's stdout, or an error once the deadline passes
        buf = b""
        fd = p.stdout.fileno()
        while not buf.endswith(b"\n"):
            left = deadline - time.time()
            if left <= 0 or not select.select([fd], [], [], left)[0]:
                raise RuntimeError("plain rank timed out")
            chunk = os.read(fd, 1)
            if not chunk:
                raise RuntimeError(f"plain rank exited with code {p.wait()}")
            buf += chunk
        return buf

    out = []
    try:
        for r in range(R):
            with open(os.path.join(tmp, f"{r}.in"), "wb") as f:
                for _, (A, B) in specs[r]:
                    f.write(np.ascontiguousarray(A, dtype=np.float32).tobytes())
                    f.write(np.ascontiguousarray(B, dtype=np.float32).tobytes())
        t_spawn = time.perf_counter()
        for r in range(R):
            core = cores[r % len(cores)] if cores else -1
            procs.append(subprocess.Popen(
                [exe, str(per_rank), str(m), str(n), str(k), os.path.join(tmp, f"{r}.in"),
                 os.path.join(tmp, f"{r}.out"), str(core), init]
                + [f"{path_no[p]}:{mode}" for p, mode in phases],
                stdin=subprocess.PIPE, stdout=subprocess.PIPE))
        ready = []
        for p in procs:
            f = readline(p).split()
            if len(f) != 4 or f[0] != b"ready":
                raise RuntimeError("plain rank did not get ready")
            ready.append((time.perf_counter() - t_spawn, int(f[1]) / 1e9, int(f[2]) / 1e9, int(f[3]) / 1e9))
        for i, (path, mode) in enumerate(phases):
            for p in procs:
                p.stdin.write(b"g")
                p.stdin.flush()
            res = []
            for p in procs:
                f = readline(p).split()
                if len(f) != 4:
                    raise RuntimeError("plain rank gave no result")
                res.append((int(f[0]), int(f[1]), int(f[2]), int(f[3])))
            bad = [r for r, x in enumerate(res) if x[3] != 0]
            if bad:
                raise RuntimeError(f"plain ranks {bad} failed with codes {[res[r][3] for r in bad]}")
            spot = []
            for r in (0, R - 1):
                spec, (A, B) = specs[r][-1]
                C = np.fromfile(os.path.join(tmp, f"{r}.out.{i}"), dtype=np.float32).reshape(m, n)
                rows = np.arange(0, m, 37)
                spot.append(oracle.rel_fro_err(C[rows], oracle.sgemm64(A[rows], B)))
            turnaround = (max(x[1] for x in res) - min(x[0] for x in res)) / 1e9
            rec = {
                "value": len(w.tasks) / turnaround,
                "unit": "tasks/s",
                "turnaround_s": turnaround,
                "parity_spot_rel_err": max(spot),
                "form": f"{R} processes (one core each), one CUDA context each, default stream, "
                        f"{'operands resident' if mode == 'resident' else 'synchronous copies per task'}, "
                        f"{'FMA' if path == 'fma' else 'split3 (fused)'} SGEMM kernel alone per task",
            }
            if init == "timed" and i == 0:
                ti = [x[2] / 1e9 for x in res]
                rec["t_init_s"] = {"mean": statistics.mean(ti), "max": max(ti),
                                   "kind": "context creation + device allocation + page-locking per process, "
                                           "all processes at once, inside the timed region"}
            out.append(rec)
        for p in procs:
            p.wait(timeout=max(1.0, deadline - time.time()))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
                p.wait()
        shutil.rmtree(tmp, ignore_errors=True)
    init_rec = None
    if init == "before":
        init_rec = {"mean_s": statistics.mean(x[1] + x[2] + x[3] for x in ready),
                    "max_s": max(x[1] + x[2] + x[3] for x in ready),
                    "context_mean_s": statistics.mean(x[1] for x in ready),
                    "alloc_mean_s": statistics.mean(x[2] for x in ready),
                    "page_lock_mean_s": statistics.mean(x[3] for x in ready),
                    "spawn_to_ready_max_s": max(x[0] for x in ready),
                    "kind": "per process, all processes initialising at once, before the start"}
    return out, init_rec


def plain_forms(w, out):
    """The plain per-rank forms beside the shared ones, like for like: the
    resident plain form against ``value`` (operands in HBM on both sides),
    the copying plain form against ``e2e`` (host buffers on both sides), the
    copying form with T_init inside its timed region (Eq. 1 as the paper
    states it), and the FMA kernel on both sides. One set of processes runs
    the four forms whose initialisation comes before the start; a second
    set, the one that initialises inside the timed region."""
    inputs = gen_inputs(w)
    phases = [("split3", "resident"), ("split3", "copy"), ("fma", "resident"), ("fma", "copy")]
    recs, init = plain_per_rank(w, inputs, phases, init="before")
    res = {"split3": {"resident": recs[0], "copy": recs[1]}, "fma": {"resident": recs[2], "copy": recs[3]},
           "t_init": init}
    recs, _ = plain_per_rank(w, inputs, [("split3", "copy")], init="timed")
    res["split3"]["copy_with_init"] = recs[0]
    # T_init of one process alone (this process keeps the GPU initialised)
    w1 = synth.Workload("plain_solo", 1, [synth.TaskSpec(0, 0, synth.TASK_SGEMM, n=512, m=512, k=512,
                                                         seed=synth.task_seed(0, 0))])
    _, solo = plain_per_rank(w1, [inputs[0]], [("split3", "resident")], init="before")
    res["t_init_one_process"] = {k: solo[k] for k in ("mean_s", "context_mean_s", "alloc_mean_s", "page_lock_mean_s")}
    ratios = {"shared_over_plain_resident": out["value"] / res["split3"]["resident"]["value"]}
    if out.get("e2e"):
        ratios["shared_e2e_over_plain_copy"] = out["e2e"]["value"] / res["split3"]["copy"]["value"]
        ratios["shared_e2e_over_plain_copy_with_init"] = (out["e2e"]["value"]
                                                          / res["split3"]["copy_with_init"]["value"])
    if out.get("fma"):
        ratios["fma_shared_over_plain_resident"] = out["fma"]["value"] / res["fma"]["resident"]["value"]
    res["ratios"] = ratios
    return res


# --------------------------------------------------------------- serving loop


def _open_loop(mgr, w, depth, vin, gin, outs):
    """Every rank of w as a native thread (gvm_open_loop_run): at each task's
    scheduled arrival it submits (host mode), keeping at most `depth` of its
    tasks in flight, and reaps completions as they come. Returns (span
    seconds from the start to the last completion, latencies in seconds =
    completion seen by the rank minus scheduled arrival, host-link bytes).

    vin = (a, b) page-locked vector operands at least as long as the longest
    vector task; gin(side) -> (A, B) page-locked operands for a square SGEMM;
    outs[r][slot] a page-locked output buffer big enough for the rank's tasks
    (task i of a rank writes slot i mod depth: with at most depth in flight,
    the slot's previous task has completed).
    """
    import paper_1511_07658_gb300 as g

    R = w.ranks
    ranks = [mgr.attach(r) for r in range(R)]
    by_rank = w.by_rank()
    arrays, arrivals, moved = [], [], 0
    for r in range(R):
        lst = by_rank[r]
        arr = (g.GvmTask * max(len(lst), 1))()
        for i, spec in enumerate(lst):
            t = arr[i]
            out = outs[r][i % depth]
            if spec.kind == synth.TASK_VADD:
                t.type, t.n = g.GVM_TASK_VADD, spec.n
                t.a, t.b, t.c = vin[0].data_ptr(), vin[1].data_ptr(), out.data_ptr()
                moved += 12 * spec.n
            else:
                A, B = gin(spec.m)
                t.type, t.m, t.n, t.k = g.GVM_TASK_SGEMM, spec.m, spec.n, spec.k
                t.a, t.b, t.c = A.data_ptr(), B.data_ptr(), out.data_ptr()
                moved += 12 * spec.m * spec.m
        arrays.append(arr if lst else (g.GvmTask * 0)())
        arrivals.append([int(spec.arrival_s * 1e9) for spec in lst])
    span, lat = mgr.open_loop_run(ranks, arrays, arrivals, max_inflight=depth)
    for rk in ranks:
        rk.detach()
    return span, sorted(x for l in lat for x in l), moved


def _lat_summary(runs):
    """Per-run latency percentiles (us) and their spread over repeated runs."""
    out = {}
    for q, name in ((50, "p50"), (99, "p99"), (99.9, "p999")):
        vals = [1e6 * percentile(lat, q) for lat in runs]
        out[name] = {"median": statistics.median(vals), "min": min(vals), "max": max(vals)}
    out["kind"] = "scheduled arrival -> completion seen by the rank; median, min and max over repeated runs"
    return out


def _load_points(run_w, make_w, capacity, fracs, repeats, extra=None):
    """Runs the workload make_w(frac) `repeats` times at each offered load
    (fraction of capacity), plus the named extra workloads; returns one
    record per point: offered and served tasks/s, latency spread."""
    points = {}
    todo = [(f"at_{f}_capacity", f, make_w(f)) for f in fracs] + list(extra or [])
    for name, frac, w1 in todo:
        spans, lats, moved = [], [], 0
        for _ in range(repeats):
            span1, lat1, moved, st1 = run_w(w1)
            if st1["device_status"]:
                raise RuntimeError(f"device status {st1['device_status']} at {name}")
            spans.append(span1)
            lats.append(lat1)
        last_arrival = max(t.arrival_s for t in w1.tasks)
        points[name] = {
            "offered_tasks_per_s": len(w1.tasks) / last_arrival if last_arrival > 0 else None,
            "offered_fraction_of_capacity": frac,
            "served_tasks_per_s": [len(w1.tasks) / x for x in spans],
            "tasks": len(w1.tasks), "last_arrival_s": last_arrival, "repeats": repeats,
            "latency_us": _lat_summary(lats),
            "host_link_gbs": moved / statistics.median(spans) / 1e9,
        }
    return points


def serving_arm(args):
    """Open-loop serving: 16 ranks, 4096 tasks, Poisson arrivals with a mean
    gap of 20 us per rank, half vector adds (n = floor(2^(16+8u))) and half
    square SGEMMs (side from {256, 512, 1024, 2048}), admission capped at
    32 GiB of device buffers. The manager runs in continuous mode: tasks are
    admitted as ring slots and staging space free up while others run.

    Ranks run as native threads (gvm_open_loop_run). Latency of a task = the
    moment its rank observes completion minus its scheduled arrival time (so
    a rank that falls behind does not hide queueing delay). First the
    capacity (every task arrives at once; tasks/s over the run), then the same
    tasks paced at 0.5 and 0.8 x capacity and at the configured 20 us gap
    (an overload), each point run `--repeats` times for the spread. Operands:
    per size, one seeded input set shared by every task of that size (the
    latency and throughput do not depend on values; parity of the mix is
    covered by the GPU tests); outputs go to per-rank pinned buffers, one per
    in-flight slot.
    """
    import torch

    import paper_1511_07658_gb300 as g

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    total = args.serving_tasks or 4096
    R = 16
    w = synth.serving_mix(ranks=R, total=total)
    depth = 8
    vmax = max(t.n for t in w.tasks if t.kind == synth.TASK_VADD)
    a, b = synth.vadd_inputs(4242, vmax)
    va, vb = torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory()
    sides = sorted({t.m for t in w.tasks if t.kind == synth.TASK_SGEMM})
    gin = {}
    for sd in sides:
        A, B = synth.sgemm_inputs(9000 + sd, sd, sd, sd)
        gin[sd] = (torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory())
    out_elems = max(vmax, max(sd * sd for sd in sides))
    outs = [[torch.empty(out_elems).pin_memory() for _ in range(depth)] for _ in range(R)]
    smax = max(sd for sd in sides)
    per_task = max(12 * vmax, 12 * smax * smax + g.sgemm_scratch_bytes(smax, smax, smax, args.path)) + (1 << 20)

    def run_w(w1):
        mgr = g.Manager(R, ring_depth=depth, mode="continuous", sgemm_path=args.path,
                        slice_bytes=per_task * 2 + (64 << 20), admission_cap_bytes=32 << 30,
                        ingest_quantum=args.quantum)
        try:
            span, lat, moved = _open_loop(mgr, w1, depth, (va, vb), lambda sd: gin[sd], outs)
            st = mgr.stats()
        finally:
            mgr.shutdown()
        return span, lat, moved, st

    w_cap = synth.serving_mix(ranks=R, total=total, gap_us=1e-6)
    cap_runs = [run_w(w_cap) for _ in range(args.repeats)]
    capacity = statistics.median(total / x[0] for x in cap_runs)
    moved = cap_runs[0][2]

    def make_w(frac):  # mean gap per rank for an offered total rate of frac x capacity
        return synth.serving_mix(ranks=R, total=total, gap_us=1e6 * R / (frac * capacity))

    points = _load_points(run_w, make_w, capacity, (0.5, 0.8), args.repeats,
                          extra=[("configured_20us_gap", None, w)])
    cfgd = points["configured_20us_gap"]
    cfgd["offered_fraction_of_capacity"] = cfgd["offered_tasks_per_s"] / capacity
    return {
        "metric": METRIC + " (serving loop)",
        "value": capacity,
        "unit": "tasks/s",
        "n_gpus": 1,
        "higher_is_better": True,
        "dtype": "bf16x3->f32" if args.path != "fma" else "f32",
        "data": "synthetic",
        "config": {"workload": f"serving mix: 16 ranks, {total} tasks, Poisson 20 us mean gap per rank, "
                   "50/50 vector add n~2^(16+8u) / square SGEMM {256,512,1024,2048}, cap 32 GiB",
                   "mode": "continuous", "sgemm_path": args.path, "ring_depth": depth,
                   "repeats": args.repeats},
        "capacity": {"tasks_per_s": capacity, "runs_tasks_per_s": [total / x[0] for x in cap_runs],
                     "host_link_gbs": moved / statistics.median(x[0] for x in cap_runs) / 1e9,
                     "kind": "every task arrives at once; tasks over the time to the last completion"},
        **points,
    }


def stress_arm(args):
    """Open-loop stress (the lognormal mix): 128 ranks, 70% vector add with n
    = round(2^20 e^(1.5 Z)) and 30% square SGEMM with side round(768
    e^(0.7 Z)) in [64, 4096], Poisson arrivals, admission capped at 120 GiB,
    continuous mode. Vector lengths are clamped to [2^10, 2^24] here: the
    manager gives every rank an equal slice of the device arena, and a 2^28
    vector add stages 3 GiB, so 128 ranks holding one each would need 384
    GiB of HBM. First the capacity: 48 tasks a rank, every task arriving at
    once (tasks/s over the whole run). Then, at 0.5, 0.8 and 0.95 x that
    capacity, Poisson arrivals for `--duration` seconds (the task count per
    rank follows from the rate), each point run `--repeats` times, with
    p50/p99/p999 latency. Operands come from one seeded page-locked buffer per
    kind (a task reads a prefix of it as a dense operand); outputs share a
    pool of page-locked buffers, one per rank slot group (values are not
    checked here; the mix's parity is covered by the GPU tests)."""
    import torch

    import paper_1511_07658_gb300 as g

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    R, P, depth = 128, args.per_rank or 48, 2

    def clamp(w):  # the clamp of this leg
        for t in w.tasks:
            if t.kind == synth.TASK_VADD:
                t.n = min(t.n, 1 << 24)
        return w

    w0 = clamp(synth.stress_mix(ranks=R, per_rank=P, rate_per_rank_hz=1e9))
    vmax = 1 << 24
    smax = 4096
    a, b = synth.vadd_inputs(5151, vmax)
    vin = (torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory())
    A, B = synth.sgemm_inputs(6161, smax, smax, smax)
    gA, gB = torch.from_numpy(A).reshape(-1).pin_memory(), torch.from_numpy(B).reshape(-1).pin_memory()
    out_elems = max(vmax, smax * smax)
    pool = [torch.empty(out_elems).pin_memory() for _ in range(16)]
    outs = [[pool[(r * depth + s) % len(pool)] for s in range(depth)] for r in range(R)]
    per_task = max(12 * vmax, 12 * smax * smax) + (1 << 20)

    def run_w(w):
        mgr = g.Manager(R, ring_depth=depth, mode="continuous", sgemm_path=args.path,
                        slice_bytes=per_task * depth + (16 << 20), admission_cap_bytes=120 << 30,
                        ingest_quantum=args.quantum)
        try:
            span, lat, moved = _open_loop(mgr, w, depth, vin, lambda sd: (gA, gB), outs)
            st = mgr.stats()
        finally:
            mgr.shutdown()
        return span, lat, moved, st

    span0, _, moved0, _ = run_w(w0)
    capacity = len(w0.tasks) / span0

    def make_w(frac):
        rate = frac * capacity / R
        per = max(1, int(math.ceil(rate * args.duration)))
        return clamp(synth.stress_mix(ranks=R, per_rank=per, rate_per_rank_hz=rate))

    points = _load_points(run_w, make_w, capacity, (0.5, 0.8, 0.95), args.repeats)
    return {
        "metric": METRIC + " (stress loop)",
        "value": capacity,
        "unit": "tasks/s",
        "n_gpus": 1,
        "higher_is_better": True,
        "dtype": "bf16x3->f32" if args.path != "fma" else "f32",
        "data": "synthetic",
        "config": {"workload": f"stress mix: {R} ranks, 70% vector add n = 2^20 e^(1.5Z) in "
                   "[2^10, 2^24], 30% square SGEMM side 768 e^(0.7Z) in [64, 4096], cap 120 GiB",
                   "mode": "continuous", "sgemm_path": args.path, "ring_depth": depth,
                   "arrivals_s_per_point": args.duration, "repeats": args.repeats},
        "capacity": {"tasks_per_s": capacity, "host_link_gbs": moved0 / span0 / 1e9, "seconds": span0,
                     "tasks": len(w0.tasks)},
        **points,
    }


class c_uint64_holder(ctypes.c_uint64):
    pass


# --------------------------------------------------------------- model check


def model_check(args, w):
    """Measured shared time against the execution model (Section 4.2.3).

    T_in, T_out: one task's input / output copy alone (pinned host memory,
    CUDA events). T_comp: the task kernel alone. Shared: N ranks, one task
    each, through the manager (host buffers), N = 1, 2, 4, 8, 16, as the
    paper's validation varies the process count (Section 6). Predictions:
    Eq. 2 or Eq. 7 by the task's class, and the duplex, wave-aware variant.
    """
    import torch

    import paper_1511_07658_gb300 as g
    from oracle import model

    spec = w.tasks[0]
    reps = 20
    if spec.kind == synth.TASK_SGEMM:
        m, n, k = spec.m, spec.n, spec.k
        hin = [torch.randn(m, k).pin_memory(), torch.randn(k, n).pin_memory()]
        hout = torch.empty(m, n).pin_memory()
    else:
        hin = [torch.randn(spec.n).pin_memory(), torch.randn(spec.n).pin_memory()]
        hout = torch.empty(spec.n).pin_memory()
    din = [x.cuda() for x in hin]
    dout = torch.empty_like(hout, device="cuda")
    s = torch.cuda.Stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            fn()
            torch.cuda.synchronize()
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    t_in = timed(lambda: [d.copy_(h, non_blocking=True) for d, h in zip(din, hin)])
    t_out = timed(lambda: hout.copy_(dout, non_blocking=True))
    if spec.kind == synth.TASK_SGEMM:
        scratch = torch.empty(g.sgemm_scratch_bytes(m, n, k, args.path) + 256, dtype=torch.uint8, device="cuda")
        t_comp = timed(lambda: g.sgemm_f32(din[0], din[1], dout, path=args.path, scratch=scratch, stream=s))
    else:
        t_comp = timed(lambda: g.vadd_f32(din[0], din[1], dout, stream=s))
    cls = model.classify(t_in, t_comp, t_out)
    # Tiles of one task in the scheduler (one CTA per SM runs them): 128 x 256
    # for split3, 128 x 128 for the FMA path; a vector task is one wave.
    if spec.kind == synth.TASK_SGEMM:
        tn = 128 if args.path == "fma" else 256
        tiles = -(-spec.m // 128) * -(-spec.n // tn)
    else:
        tiles = 1
    rows = []
    for N in (1, 2, 4, 8, 16):
        mgr = g.Manager(N, ring_depth=4, sgemm_path=args.path, slice_bytes=64 << 20)
        ranks = [mgr.attach(r) for r in range(N)]
        outs = [torch.empty_like(hout).pin_memory() for _ in range(N)]

        def step():
            seqs = []
            for r in range(N):
                if spec.kind == synth.TASK_SGEMM:
                    seqs.append(ranks[r].submit_sgemm(hin[0], hin[1], outs[r]))
                else:
                    seqs.append(ranks[r].submit_vadd(hin[0], hin[1], outs[r]))
            mgr.flush()
            for r in range(N):
                ranks[r].sync(seqs[r])

        for _ in range(3):
            step()
        t0 = time.perf_counter()
        for _ in range(reps):
            step()
        shared = (time.perf_counter() - t0) / reps
        mgr.shutdown()
        pred = model.shared_time(N, t_in, t_comp, t_out)
        rows.append({
            "N": N,
            "measured_s": shared,
            "eq2_or_eq7_s": pred,
            "deviation": model.deviation(shared, pred),
            "duplex_s": model.shared_time_duplex(N, t_in, t_comp, t_out, model.waves(N, tiles, GB300_SMS, 1)),
            "eq1_no_init_s": model.t_total_no_vt(N, 0.0, t_in, t_comp, t_out, 0.0),
        })
    return {"t_in_s": t_in, "t_comp_s": t_comp, "t_out_s": t_out, "class": cls, "rows": rows,
            "mean_deviation": statistics.mean(r["deviation"] for r in rows)}


def paper_ps_check():
    """The paper's own mechanism and model (Sections 4.2.1-4.2.3, Section 6):
    N ranks of one manager in GVM_MODE_PS1 or GVM_MODE_PS2 each submit one
    host-mode task; gvm_flush (the request barrier) issues every task's
    copies and kernel on its rank's stream in the style's order. The shared
    time (first issue to the last rank's completion, CUDA events on the rank
    streams) for N = 1, 2, 4, 8, 16 against Eqs. 2-7 from solo T_in, T_comp,
    T_out, profiled first with the same copies and kernel on one stream, as
    the paper derives them. Cases: compute-intensive FMA SGEMM 2048^3 (fills
    the GPU) and a one-CTA FMA SGEMM 128 x 128 x 16384 (leaves the other SMs
    free, as the model's full kernel overlap assumes, like the paper's one-
    block EP kernel); I/O-intensive vector add and vector multiply with 15
    products (Table 2), n = 2^24 each. Deviation as Section 6 reports it."""
    import torch

    import paper_1511_07658_gb300 as g
    from oracle import model

    reps = 5
    nmax = 16
    out = {}
    cases = {
        "ci_sgemm_fma_2048": ("sgemm", (2048, 2048, 2048)),
        "ci_sgemm_fma_1cta_128x128x16384": ("sgemm", (128, 128, 16384)),
        "ioi_vadd_2p24": ("vadd", 1 << 24),
        "ioi_vmul_2p24_x15": ("vmul", 1 << 24),
    }
    for name, (kind, size) in cases.items():
        if kind == "sgemm":
            mm, nn, kk = size
            hin = [[torch.randn(mm, kk).pin_memory(), torch.randn(kk, nn).pin_memory()] for _ in range(nmax)]
            hout = [torch.empty(mm, nn).pin_memory() for _ in range(nmax)]
        elif kind == "vmul":
            hin = [[torch.rand(size).pin_memory(), (0.75 + 0.5 * torch.rand(size)).pin_memory()] for _ in range(nmax)]
            hout = [torch.empty(size).pin_memory() for _ in range(nmax)]
        else:
            hin = [[torch.randn(size).pin_memory(), torch.randn(size).pin_memory()] for _ in range(nmax)]
            hout = [torch.empty(size).pin_memory() for _ in range(nmax)]
        task_bytes = sum(x.numel() * 4 for x in hin[0]) + hout[0].numel() * 4

        # ---- solo profile: one stream, the task's copies and kernel alone
        din = [x.cuda() for x in hin[0]]
        dout = torch.empty_like(hout[0], device="cuda")
        st = torch.cuda.Stream()

        def h2d():
            for d, h in zip(din, hin[0]):
                d.copy_(h, non_blocking=True)

        def comp():
            if kind == "sgemm":
                g.sgemm_f32(din[0], din[1], dout, path="fma", stream=st)
            elif kind == "vmul":
                g.vmul_f32(din[0], din[1], dout, 15, stream=st)
            else:
                g.vadd_f32(din[0], din[1], dout, stream=st)

        def d2h():
            hout[0].copy_(dout, non_blocking=True)

        def solo(fn):
            times = []
            for _ in range(reps + 2):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(st):
                    e0.record(st)
                    fn()
                    e1.record(st)
                e1.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
            return statistics.median(times[2:])

        t_in, t_comp, t_out = solo(h2d), solo(comp), solo(d2h)
        del din, dout
        torch.cuda.empty_cache()

        # ---- shared: the manager in PS-1 / PS-2 mode
        def shared_times(style):
            mgr = g.Manager(nmax, ring_depth=2, mode=f"ps{style}", sgemm_path="fma",
                            slice_bytes=(task_bytes + (8 << 20)) // (1 << 20) * (1 << 20) + (1 << 20))
            ranks = [mgr.attach(r) for r in range(nmax)]

            def submit(r):
                a, b = hin[r]
                if kind == "sgemm":
                    return ranks[r].submit_sgemm(a, b, hout[r])
                if kind == "vmul":
                    return ranks[r].submit_vmul(a, b, hout[r], 15)
                return ranks[r].submit_vadd(a, b, hout[r])

            def run(n):
                torch.cuda.synchronize()
                cur = torch.cuda.current_stream()
                seqs = [submit(r) for r in range(n)]  # the ranks' requests; nothing is issued yet
                e0 = torch.cuda.Event(enable_timing=True)
                e0.record(cur)
                for r in range(n):
                    mgr.copy_streams[2 * r].wait_event(e0)
                mgr.flush()
                for r in range(n):
                    ev = torch.cuda.Event()
                    ev.record(mgr.copy_streams[2 * r])
                    cur.wait_event(ev)
                e1 = torch.cuda.Event(enable_timing=True)
                e1.record(cur)
                e1.synchronize()
                for r in range(n):
                    ranks[r].sync(seqs[r])
                return e0.elapsed_time(e1) / 1e3

            res = {}
            for n in (1, 2, 4, 8, 16):
                run(n)
                res[n] = statistics.median(run(n) for _ in range(reps))
            mgr.shutdown()
            return res

        meas = {1: shared_times(1), 2: shared_times(2)}
        rows = []
        for n in (1, 2, 4, 8, 16):
            row = {"N": n}
            for style in (1, 2):
                if style == 1:
                    pred = model.t_total_ci_ps1(n, t_in, t_comp, t_out)  # Eq. 2 = Eq. 4
                else:
                    pred = (model.t_total_ci_ps2(n, t_in, t_comp, t_out) if model.classify(t_in, t_comp, t_out) == model.CI
                            else model.t_total_ioi_ps2(n, t_in, t_comp, t_out))  # Eq. 3 or Eq. 7
                row[f"ps{style}_measured_s"] = meas[style][n]
                row[f"ps{style}_model_s"] = pred
                row[f"ps{style}_deviation"] = model.deviation(meas[style][n], pred)
            row["eq1_no_init_s"] = model.t_total_no_vt(n, 0.0, t_in, t_comp, t_out, 0.0)
            rows.append(row)
        out[name] = {
            "t_in_s": t_in, "t_comp_s": t_comp, "t_out_s": t_out, "class": model.classify(t_in, t_comp, t_out),
            "rows": rows,
            "mean_deviation_ps1": statistics.mean(r["ps1_deviation"] for r in rows),
            "mean_deviation_ps2": statistics.mean(r["ps2_deviation"] for r in rows),
            # Section 6 validates with N = 1..8
            "mean_deviation_ps1_n1to8": statistics.mean(r["ps1_deviation"] for r in rows if r["N"] <= 8),
            "mean_deviation_ps2_n1to8": statistics.mean(r["ps2_deviation"] for r in rows if r["N"] <= 8),
        }
        del hin, hout
    return out


def overhead_check():
    """Virtualization-layer overhead (Section 6): one rank, one vector add of
    1 MB to 400 MB per operand array through the manager (host buffers,
    submit -> flush -> sync on the host clock) against the same copies and
    kernel issued directly on one stream (CUDA events): (turnaround - direct)
    / direct per size."""
    import torch

    import paper_1511_07658_gb300 as g

    rows = []
    for mb in (1, 4, 16, 64, 256, 400):
        n = mb * (1 << 20) // 4
        a = torch.rand(n).pin_memory()
        b = torch.rand(n).pin_memory()
        c = torch.empty(n).pin_memory()
        da, db, dc = a.cuda(), b.cuda(), torch.empty(n, device="cuda")
        st = torch.cuda.Stream()

        def direct():
            with torch.cuda.stream(st):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                da.copy_(a, non_blocking=True)
                db.copy_(b, non_blocking=True)
                g.vadd_f32(da, db, dc, stream=st)
                c.copy_(dc, non_blocking=True)
                e1.record(st)
            e1.synchronize()
            return e0.elapsed_time(e1) / 1e3

        for _ in range(2):
            direct()
        t_direct = statistics.median(direct() for _ in range(5))
        mgr = g.Manager(1, ring_depth=2, slice_bytes=3 * 4 * n + (8 << 20))
        rk = mgr.attach(0)

        def managed():
            t0 = time.perf_counter()
            seq = rk.submit_vadd(a, b, c)
            mgr.flush()
            rk.sync(seq)
            return time.perf_counter() - t0

        for _ in range(2):
            managed()
        t_mgr = statistics.median(managed() for _ in range(5))
        mgr.shutdown()
        rows.append({"mb_per_array": mb, "direct_s": t_direct, "manager_s": t_mgr,
                     "overhead": (t_mgr - t_direct) / t_direct})
        del a, b, c, da, db, dc
    return {"rows": rows, "kind": "one rank, host buffers; direct = copies + kernel on one stream"}


# --------------------------------------------------------------- grouped


def grouped_arm(args):
    """Batching config: R ranks x P SGEMM tasks, M, N, K each drawn from
    {128, 192, ..., 2048}, all in one persistent scheduler launch per step.

    Operands are resident and drawn on the device (seeded torch generator):
    per rank one 2048 x 2048 pool for A and one for B; task i multiplies the
    leading m x k block of A's pool (every prefix of a row-major block is a
    row-major m x k matrix) by the leading k x n block of B's pool into its
    own C. Inputs of the full config would not fit the host's generator in
    minutes (about 233 GB); this keeps every shape and every byte of C
    distinct while reusing operand memory. Sampled rows of three tasks are
    checked against the binary64 oracle."""
    import torch

    import oracle
    import paper_1511_07658_gb300 as g

    torch.cuda.set_device(0)
    R, P = args.ranks or 64, args.per_rank or 256
    w = synth.grouped_mixed(ranks=R, per_rank=P)
    side = 2048
    pool = 4 * side * side

    def al256(x):
        return (x + 255) // 256 * 256

    c_off = {}
    need = [2 * pool] * R
    for spec in w.tasks:
        c_off[(spec.rank, spec.index)] = need[spec.rank]
        need[spec.rank] += al256(4 * spec.m * spec.n)
    resident = max(need)
    mgr = g.Manager(R, ring_depth=max(2, 1 << (P - 1).bit_length()), mode="barrier", sgemm_path=args.path,
                    slice_bytes=resident + (4 << 20), resident_bytes=resident, ingest_quantum=args.quantum,
                    l2_prefetch=None if args.l2_prefetch is None else bool(args.l2_prefetch))
    ranks = [mgr.attach(r) for r in range(R)]
    gen = torch.Generator(device="cuda")
    for r in range(R):
        gen.manual_seed(synth.task_seed(r, 0))
        v = ranks[r].resident_view(0, (2, side * side))
        v.copy_(torch.randn(2, side * side, generator=gen, device="cuda"))
    arrays = []
    by_rank = [[s for s in w.tasks if s.rank == r] for r in range(R)]
    for r in range(R):
        arr = (g.GvmTask * P)()
        for i, spec in enumerate(by_rank[r]):
            t = arr[i]
            t.type, t.flags = g.GVM_TASK_SGEMM, g.GVM_TASK_RESIDENT
            t.m, t.n, t.k = spec.m, spec.n, spec.k
            t.a_off, t.b_off, t.c_off = 0, pool, c_off[(r, spec.index)]
        arrays.append(arr)
    flops = sum(2.0 * s.m * s.n * s.k for s in w.tasks)
    torch.cuda.synchronize()
    mgr.spmd_run(ranks, arrays, args.warmup)
    sampler = ClockSampler(0)
    torch.cuda.synchronize()
    sampler.start()
    st0 = torch.cuda.Event(enable_timing=True)
    st1 = torch.cuda.Event(enable_timing=True)
    st0.record(mgr.sched_stream)
    dev, launch, _ = mgr.spmd_run(ranks, arrays, args.steps)
    st1.record(mgr.sched_stream)
    torch.cuda.synchronize()
    sampler.stop()
    total_s = st0.elapsed_time(st1) / 1e3
    kmean = statistics.mean(launch) / 1e3
    st = mgr.stats()
    ph = st["launch_phase"]
    # parity: sampled rows of three tasks against the binary64 oracle
    errs = []
    for r, i in ((0, 0), (R - 1, P - 1), (R // 2, P // 3)):
        spec = by_rank[r][i]
        A = ranks[r].resident_view(0, (spec.m, spec.k)).cpu().numpy()
        B = ranks[r].resident_view(pool, (spec.k, spec.n)).cpu().numpy()
        C = ranks[r].resident_view(c_off[(r, spec.index)], (spec.m, spec.n)).cpu().numpy()
        rows = np.arange(0, spec.m, 29)
        errs.append(float(oracle.rel_fro_err(C[rows], oracle.sgemm64(A[rows], B))))
    mgr.shutdown()
    pk, pk_kind = peaks()
    # A launch this long runs back to back under the power cap: the measured
    # sustained bf16 rate is its peak (the burst one for short launches),
    # with the burst fraction kept beside it.
    sustained = kmean >= 0.05 and "bf16_tflops_sustained" in pk
    burst_frac = None
    if args.path != "fma":
        tf = pk["bf16_tflops_sustained"] if sustained else pk["bf16_tflops"]
        peak = tf / 3.0
        basis = f"bf16 dense {tf} TFLOP/s ({pk_kind}, {'sustained' if sustained else 'burst'}) / 3 products"
        bound = "tensor"
        burst_frac = flops / kmean / 1e12 / (pk["bf16_tflops"] / 3.0)
    else:
        peak = GB300_SMS * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        basis = "152 SMs x 128 FP32 lanes x 2 flop x max SM clock"
        bound = "alu"
    achieved = flops / kmean / 1e12
    return {
        "metric": METRIC + " (grouped mixed shapes)",
        "value": len(w.tasks) * args.steps / total_s,
        "unit": "tasks/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True,
        "dtype": "bf16x3->f32" if args.path != "fma" else "f32",
        "data": "synthetic",
        "config": {"workload": f"grouped SGEMM: {R} ranks x {P} tasks, M, N, K each from {{128..2048}} step 64, "
                               "standard-normal operands drawn on the device, resident",
                   "sgemm_path": args.path, "mode": "barrier", "tflop_per_step": flops / 1e12},
        "roofline": {"bound": bound, "unit": "TFLOP/s", "achieved": achieved, "peak": peak, "frac": achieved / peak,
                     "peak_basis": basis, "frac_of_burst_peak": burst_frac,
                     "kernel": "gvm::" + {"split3": "sched_fused_kernel",
                                          "split3_wide": "sched_wide_kernel",
                                          "split3_tma": "sched_tma_kernel"}.get(args.path, "sched_fma_kernel"),
                     "traffic": ncu_traffic({"split3": "sched_fused_kernel", "split3_wide": "sched_wide_kernel",
                                             "split3_tma": "sched_tma_kernel"}.get(
                         args.path, "sched_fma_kernel") + "/grouped") if (R, P) == (64, 256) else None,
                     "launch_ms": kmean * 1e3},
        "sched_timeline_last_launch": {
            "cta_ms": {"acquire": ph[0] / 1e6, "stage_wait": ph[2] / 1e6, "gemm": ph[3] / 1e6,
                       "mma_wait": ph[4] / 1e6, "epilogue": ph[8] / 1e6},
            "tiles": ph[6]},
        "parity_spot_rel_err": max(errs),
        "clocks": sampler.summary(),
        "device_status": st["device_status"],
    }


# --------------------------------------------------------------- main


def main():
    args = parse()
    if args.path is None:  # the split3 tile form the autotuner chose for this workload class (fused if none)
        from paper_1511_07658_gb300.manager import tuning

        t = tuning()
        args.path = (t.get("sgemm_form_by_class", {}).get("grouped") if args.workload == "grouped" else None) \
            or t.get("sgemm_form", "split3")
    if args.ipc_client:
        ipc_client_main(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.workload == "grouped":
        if args.impl == "reference" or rank != 0:
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the grouped config has no CPU reference arm"}))
            return
        print(json.dumps(grouped_arm(args)))
        return
    if args.workload == "stress":
        if args.impl == "reference" or rank != 0:
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the stress loop has no CPU reference arm"}))
            return
        print(json.dumps(stress_arm(args)))
        return
    if args.workload == "serving":
        if args.impl == "reference" or rank != 0:
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable": "the serving loop has no CPU reference arm"}))
            return
        print(json.dumps(serving_arm(args)))
        return
    w, desc = workload(args.workload, args.ranks, args.per_rank)
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(reference_arm(args, w, desc)))
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    out = gpu_arm(args, w, desc, rank, world)
    if rank == 0:
        extras = world == 1 and not args.skip_extra and args.workload == "sgemm512"
        if extras and args.path != "fma":
            # The plain FP32-FMA path on the same workload (the precision
            # baseline of the headline's split3 arithmetic).
            out["fma"] = resident_leg(args, w, gen_inputs(w), "fma", max(3, args.steps // 2), args.warmup, "sgemm512")
        if extras:
            # Vector adds through the scheduler at a size far beyond L2: the
            # HBM roofline of the elementwise task kernel on the product path.
            wv = synth.vadd_tiny(ranks=16, per_rank=4, n=1 << 22)
            out["vadd_hbm"] = resident_leg(args, wv, gen_inputs(wv), args.path, max(5, args.steps), args.warmup,
                                           "vadd_hbm")
            out["vadd_hbm"]["workload"] = "vector add n=2^22, 16 ranks x 4 tasks (3.2 GB of HBM traffic a step)"
        if extras and not args.skip_plain:
            out["plain_per_rank"] = plain_forms(w, out)
        if not args.skip_cpu:
            out["cpu_baseline"] = cpu_baseline(w)
        if args.cross_process:
            out["cross_process"] = cross_process_check(args, w)
        if args.model:
            out["model_check"] = model_check(args, w)
            out["paper_ps_model"] = paper_ps_check()
            out["virtualization_overhead"] = overhead_check()
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
