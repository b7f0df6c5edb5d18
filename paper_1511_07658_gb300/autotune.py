"""Autotuner of the manager's copy and tile granularity.

    python -m paper_1511_07658_gb300.autotune            # writes tuning.json

On the current GPU it times, through the native SPMD harness
(``gvm_spmd_run``), short runs of two workloads for each candidate setting
and keeps the fastest:

* ``copy_run_bytes`` (how far host-mode copies of a batch are merged): the
  end-to-end leg of 16 ranks x 16 SGEMM 512^3 tasks, each rank's operands in
  one pinned block (8 steps);
* ``vadd_tile`` (elements per vector-add tile; 0 = per task, n / CTAs): 16
  ranks x 8 resident vector adds of n = 2^22 (10 steps);
* ``sgemm_form`` (the split3 SGEMM tile form): fused 128 x 256 tiles
  (operands loaded by the staging warps), the same tiles with A and B landed
  by TMA and split in place, and wide 256 x 256 tiles of one CTA (A by TMA),
  per workload class: square 512^3 (16 x 64 tasks, the headline shape),
  512 x 768 x 512 (16 x 16), 2048^3 (16 x 1) and a grouped mix of shapes
  drawn from {128, ..., 2048} (64 ranks x 64 tasks, a quarter of the
  grouped benchmark's tasks per rank). ``sgemm_form_by_class`` keeps the
  fastest form of each class; ``sgemm_form``, the manager's default, is the
  512^3 class's. A tile form per task inside one launch would need several
  forms in one kernel, whose converters then spill (measured); so the form
  is chosen per manager (per workload), and a task's result is the same
  alone and in any mix (every form computes each element the same way);
* ``l2_prefetch`` (split3: the next queued tile's operands prefetched into
  L2): on against off on the same three workloads, kept if it wins all.

The table it writes (``tuning.json`` beside this file: the choice, the device
and every timing) is what ``Manager`` uses when the caller passes neither
setting. Inputs are seeded synthetic data drawn on the device.
"""
from __future__ import annotations

import json
import statistics
import sys

import torch

from . import manager as _m
from .manager import GVM_TASK_RESIDENT, GVM_TASK_SGEMM, GVM_TASK_VADD, GvmTask, Manager

COPY_RUNS = (4 << 20, 16 << 20, 64 << 20)
SGEMM_FORMS = ("split3", "split3_tma", "split3_wide")
VADD_TILES = (0, 1 << 16, 1 << 18, 1 << 20)


def _al(x: int) -> int:
    return (x + 255) // 256 * 256


def time_copy_run(run_bytes: int, ranks: int = 16, per_rank: int = 16, side: int = 512, steps: int = 8) -> float:
    """Median step time (s) of the end-to-end SGEMM leg."""
    la = 4 * side * side
    per_task = 3 * _al(la)
    mgr = Manager(ranks, ring_depth=per_rank, mode="barrier", sgemm_path="split3",
                  slice_bytes=per_task * per_rank + (16 << 20), copy_run_bytes=run_bytes)
    try:
        rk = [mgr.attach(r) for r in range(ranks)]
        gen = torch.Generator(device="cuda")
        gen.manual_seed(1234)
        arrays, keep = [], []
        for r in range(ranks):
            inb = torch.randn(per_rank * 2 * la // 4, generator=gen, device="cuda").cpu().pin_memory()
            outb = torch.empty(per_rank * la // 4).pin_memory()
            keep += [inb, outb]
            arr = (GvmTask * per_rank)()
            for i in range(per_rank):
                t = arr[i]
                t.type, t.flags, t.m, t.n, t.k = GVM_TASK_SGEMM, 0, side, side, side
                t.a = inb.data_ptr() + 2 * la * i
                t.b = t.a + la
                t.c = outb.data_ptr() + la * i
            arrays.append(arr)
        mgr.spmd_run(rk, arrays, 2)
        dev, _, _ = mgr.spmd_run(rk, arrays, steps)
        return statistics.median(dev) / 1e3
    finally:
        mgr.shutdown()


def time_vadd_tile(tile: int, ranks: int = 16, per_rank: int = 8, n: int = 1 << 22, steps: int = 10) -> float:
    """Median step time (s) of resident vector adds."""
    nb = 4 * n
    mgr = Manager(ranks, ring_depth=per_rank, mode="barrier", sgemm_path="split3",
                  slice_bytes=3 * nb * per_rank + (4 << 20), resident_bytes=3 * nb * per_rank, vadd_tile=tile)
    try:
        rk = [mgr.attach(r) for r in range(ranks)]
        gen = torch.Generator(device="cuda")
        gen.manual_seed(99)
        arrays = []
        for r in range(ranks):
            rk[r].resident_view(0, (2 * per_rank * n,)).copy_(
                torch.rand(2 * per_rank * n, generator=gen, device="cuda") * 2 - 1)
            arr = (GvmTask * per_rank)()
            for i in range(per_rank):
                t = arr[i]
                t.type, t.flags, t.n = GVM_TASK_VADD, GVM_TASK_RESIDENT, n
                t.a_off, t.b_off = 2 * nb * i, 2 * nb * i + nb
                t.c_off = 2 * nb * per_rank + nb * i
            arrays.append(arr)
        mgr.spmd_run(rk, arrays, 2)
        dev, _, _ = mgr.spmd_run(rk, arrays, steps)
        return statistics.median(dev) / 1e3
    finally:
        mgr.shutdown()


def time_sgemm(m: int, n: int, k: int, ranks: int = 16, per_rank: int = 16, steps: int = 8,
               path: str = "split3", prefetch: bool = False) -> float:
    """Median step time (s) of resident SGEMMs, every task m x n x k."""
    la, lb, lc = 4 * m * k, 4 * k * n, 4 * m * n
    per_task = _al(la) + _al(lb) + _al(lc)
    mgr = Manager(ranks, ring_depth=max(2, 1 << (per_rank - 1).bit_length()), mode="barrier", sgemm_path=path,
                  slice_bytes=per_task * per_rank + (4 << 20), resident_bytes=per_task * per_rank,
                  l2_prefetch=prefetch)
    try:
        rk = [mgr.attach(r) for r in range(ranks)]
        gen = torch.Generator(device="cuda")
        gen.manual_seed(7)
        arrays = []
        for r in range(ranks):
            rk[r].resident_view(0, (per_task * per_rank // 4,)).copy_(
                torch.randn(per_task * per_rank // 4, generator=gen, device="cuda"))
            arr = (GvmTask * per_rank)()
            for i in range(per_rank):
                t = arr[i]
                t.type, t.flags, t.m, t.n, t.k = GVM_TASK_SGEMM, GVM_TASK_RESIDENT, m, n, k
                t.a_off = per_task * i
                t.b_off = t.a_off + _al(la)
                t.c_off = t.b_off + _al(lb)
            arrays.append(arr)
        mgr.spmd_run(rk, arrays, 2)
        dev, _, _ = mgr.spmd_run(rk, arrays, steps)
        return statistics.median(dev) / 1e3
    finally:
        mgr.shutdown()


SGEMM_SHAPES = ((512, 512, 512, 64), (512, 768, 512, 16), (2048, 2048, 2048, 1))  # m, n, k, tasks a rank
GROUPED_CLASS = "grouped"


def time_grouped(path: str, ranks: int = 64, per_rank: int = 64, steps: int = 4) -> float:
    """Median step time (s) of resident SGEMMs with M, N, K drawn from
    {128, ..., 2048} (the grouped recipe), operands drawn on the device."""
    import synth

    w = synth.grouped_mixed(ranks=ranks, per_rank=per_rank)
    side = 2048
    pool = 4 * side * side
    need, offs = [2 * pool] * ranks, {}
    for spec in w.tasks:
        offs[(spec.rank, spec.index)] = need[spec.rank]
        need[spec.rank] += _al(4 * spec.m * spec.n)
    resident = max(need)
    mgr = Manager(ranks, ring_depth=max(2, 1 << (per_rank - 1).bit_length()), mode="barrier", sgemm_path=path,
                  slice_bytes=resident + (4 << 20), resident_bytes=resident)
    try:
        rk = [mgr.attach(r) for r in range(ranks)]
        gen = torch.Generator(device="cuda")
        gen.manual_seed(5)
        arrays = []
        for r in range(ranks):
            rk[r].resident_view(0, (2 * side * side,)).copy_(torch.randn(2 * side * side, generator=gen, device="cuda"))
            arr = (GvmTask * per_rank)()
            for i, spec in enumerate(w.by_rank()[r]):
                t = arr[i]
                t.type, t.flags, t.m, t.n, t.k = GVM_TASK_SGEMM, GVM_TASK_RESIDENT, spec.m, spec.n, spec.k
                t.a_off, t.b_off, t.c_off = 0, pool, offs[(r, i)]
            arrays.append(arr)
        mgr.spmd_run(rk, arrays, 1)
        dev, _, _ = mgr.spmd_run(rk, arrays, steps)
        return statistics.median(dev) / 1e3
    finally:
        mgr.shutdown()


def _shape_key(m, n, k):
    return f"{m}x{n}x{k}"


HEADLINE_CLASS = "512x512x512"


def choose_sgemm(form_t: dict, pf_t: dict) -> dict:
    """Per workload class the faster tile form; the manager's default is the
    headline class's (512^3). The prefetch is kept only if it wins every
    workload timed (step times in seconds, keyed by shape)."""
    by_class = {c: min(t, key=t.get) for c, t in form_t.items()}
    pf = all(t["1"] < t["0"] for t in pf_t.values())
    return {"sgemm_form": by_class[HEADLINE_CLASS], "sgemm_form_by_class": by_class, "l2_prefetch": int(pf)}


def run(path: str = _m.TUNING_FILE) -> dict:
    torch.cuda.set_device(0)
    copy_t = {str(c): time_copy_run(c) for c in COPY_RUNS}
    vadd_t = {str(v): time_vadd_tile(v) for v in VADD_TILES}
    form_t, pf_t = {}, {}
    for m, n, k, per in SGEMM_SHAPES:
        key = _shape_key(m, n, k)
        form_t[key] = {f: time_sgemm(m, n, k, per_rank=per, path=f) for f in SGEMM_FORMS}
        pf_t[key] = {str(int(on)): time_sgemm(m, n, k, per_rank=per, prefetch=on) for on in (False, True)}
    form_t[GROUPED_CLASS] = {f: time_grouped(f) for f in SGEMM_FORMS}
    choice = {
        "copy_run_bytes": int(min(copy_t, key=copy_t.get)),
        "vadd_tile": int(min(vadd_t, key=vadd_t.get)),
        **choose_sgemm(form_t, pf_t),
    }
    out = {
        "device": torch.cuda.get_device_name(0),
        "choice": choice,
        "step_s": {"copy_run_bytes": copy_t, "vadd_tile": vadd_t, "sgemm_form": form_t, "l2_prefetch": pf_t},
        "workloads": {
            "copy_run_bytes": "end-to-end leg, 16 ranks x 16 SGEMM 512^3, operands in one pinned block per rank",
            "vadd_tile": "16 ranks x 8 resident vector adds, n = 2^22",
            "sgemm_form": "resident SGEMM, 16 ranks x (64 of 512^3, 16 of 512 x 768 x 512, 1 of 2048^3), "
                          "64 ranks x 64 of the grouped mix: fused 128 x 256 tiles, the same tiles landed by TMA, "
                          "wide 256 x 256 tiles",
            "l2_prefetch": "the same SGEMM workloads, fused tiles, next-tile L2 prefetch off (0) and on (1)",
        },
    }
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    return out


if __name__ == "__main__":
    print(json.dumps(run(sys.argv[1] if len(sys.argv) > 1 else _m.TUNING_FILE), indent=1))
