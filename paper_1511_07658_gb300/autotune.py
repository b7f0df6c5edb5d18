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
* ``sgemm_tile_cost`` (the split3 SGEMM tile shape): the time of one tile
  128 x w for each width w in 128, 192, 256, from resident SGEMMs whose n
  (768) every width divides, so no tile is padded: 16 ranks x 16 tasks of
  512 x 768 x 512 at each fixed width (8 steps). The manager then gives a
  task of n columns the width minimising ceil(n / w) * cost(w), a pure
  function of the shape (a task's result is the same alone and in any mix);
* ``sgemm_form``: the same workload and the 16 x 64 SGEMM 512^3 step with
  the wide form (256 x 256 tiles of one CTA) against the fused 128-row form,
  recorded for the table; the manager's default path stays the fused form
  unless the wide one wins both.

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


TILE_WIDTHS = (128, 192, 256)


def time_sgemm(m: int, n: int, k: int, ranks: int = 16, per_rank: int = 16, steps: int = 8,
               path: str = "split3", tile_n: int | None = None) -> float:
    """Median step time (s) of resident SGEMMs, every task m x n x k."""
    la, lb, lc = 4 * m * k, 4 * k * n, 4 * m * n
    per_task = _al(la) + _al(lb) + _al(lc)
    mgr = Manager(ranks, ring_depth=per_rank, mode="barrier", sgemm_path=path,
                  slice_bytes=per_task * per_rank + (4 << 20), resident_bytes=per_task * per_rank,
                  sgemm_tile_n=tile_n)
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


def tile_costs(step_s: dict, m: int = 512, n: int = 768, tasks: int = 256) -> dict:
    """Time of one tile per width, relative to the 256-wide tile, from the
    step times of the unpadded workload (tasks x (m / 128) x (n / w) tiles)."""
    per_tile = {w: step_s[str(w)] / (tasks * (m // 128) * (n // w)) for w in TILE_WIDTHS}
    return {str(w): per_tile[w] / per_tile[256] for w in TILE_WIDTHS}


def choose_width(n: int, cost: dict) -> int:
    """The manager's rule: the width minimising ceil(n / w) * cost(w), the
    wider on ties (the same rule as the library's sgemm_tile_width)."""
    best, best_t = 256, None
    for w in sorted(TILE_WIDTHS, reverse=True):
        t = -(-n // w) * cost[str(w)]
        if best_t is None or t < best_t:
            best, best_t = w, t
    return best


def run(path: str = _m.TUNING_FILE) -> dict:
    torch.cuda.set_device(0)
    copy_t = {str(c): time_copy_run(c) for c in COPY_RUNS}
    vadd_t = {str(v): time_vadd_tile(v) for v in VADD_TILES}
    tile_t = {str(w): time_sgemm(512, 768, 512, tile_n=w) for w in TILE_WIDTHS}
    form_t = {
        "split3 512x768x512": tile_t["256"],
        "split3_wide 512x768x512": time_sgemm(512, 768, 512, path="split3_wide"),
        "split3 512^3": time_sgemm(512, 512, 512, per_rank=64),
        "split3_wide 512^3": time_sgemm(512, 512, 512, per_rank=64, path="split3_wide"),
    }
    wide_wins = (form_t["split3_wide 512x768x512"] < form_t["split3 512x768x512"]
                 and form_t["split3_wide 512^3"] < form_t["split3 512^3"])
    choice = {
        "copy_run_bytes": int(min(copy_t, key=copy_t.get)),
        "vadd_tile": int(min(vadd_t, key=vadd_t.get)),
        "sgemm_tile_cost": tile_costs(tile_t),
        "sgemm_form": "split3_wide" if wide_wins else "split3",
    }
    out = {
        "device": torch.cuda.get_device_name(0),
        "choice": choice,
        "step_s": {"copy_run_bytes": copy_t, "vadd_tile": vadd_t, "sgemm_tile_n": tile_t, "sgemm_form": form_t},
        "workloads": {
            "copy_run_bytes": "end-to-end leg, 16 ranks x 16 SGEMM 512^3, operands in one pinned block per rank",
            "vadd_tile": "16 ranks x 8 resident vector adds, n = 2^22",
            "sgemm_tile_n": "16 ranks x 16 resident SGEMM 512 x 768 x 512 at each fixed tile width",
            "sgemm_form": "fused 128-row tiles against wide 256 x 256 tiles: 16 x 16 SGEMM 512 x 768 x 512 and "
                          "16 x 64 SGEMM 512^3, resident",
        },
    }
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    return out


if __name__ == "__main__":
    print(json.dumps(run(sys.argv[1] if len(sys.argv) > 1 else _m.TUNING_FILE), indent=1))
