"""Seeded synthetic inputs for the GPU-sharing workloads.

This module is the one piece shared by the CPU oracle's harness and the CUDA
path's harness. It holds only random-number generation and workload recipes
(shapes, seeds, arrival times); none of the method's arithmetic lives here.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in its counter form: draw i of stream
``seed`` is ``mix64(seed + (i + 1) * GAMMA)``.

* ``uniform_pm1``: the top 24 bits k of a draw give ``k * 2**-23 - 1``. Every
  value is a multiple of 2**-23 in [-1, 1), exact in binary32, so a sum of two
  such values is exact or rounded once and never subnormal.
* ``standard_normal``: Box-Muller in float64 from two draws, rounded to float32.

The workloads follow the paper's benchmark shapes (Table 2: a vector addition
and a single-precision matrix multiplication, Section 6) and the five
configurations the build is measured on; see ``workload`` below.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
MASK64 = (1 << 64) - 1

TASK_VADD = 1
TASK_SGEMM = 2
TASK_VMUL = 3

_CHUNK = 1 << 22


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+n-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + idx * GAMMA
        return _mix64(z)


def splitmix64_scalar(seed: int, i: int) -> int:
    """Draw ``i`` of stream ``seed`` with Python integers (reference form)."""
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _chunked(fn, n: int, out_dtype, threads: int | None = None) -> np.ndarray:
    out = np.empty(n, dtype=out_dtype)
    if n <= _CHUNK:
        fn(0, n, out)
        return out
    starts = list(range(0, n, _CHUNK))
    workers = threads or min(16, os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(lambda s: fn(s, min(n, s + _CHUNK), out), starts))
    return out


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` float32 values k*2**-23 - 1, k = top 24 bits of each draw."""

    def fill(s, e, out):
        k = splitmix64(seed, e - s, offset + s) >> np.uint64(40)
        out[s:e] = (k.astype(np.float64) * (2.0 ** -23) - 1.0).astype(np.float32)

    return _chunked(fill, n, np.float32)


def standard_normal(seed: int, n: int) -> np.ndarray:
    """``n`` float32 standard normals; value i uses draws 2i and 2i+1."""

    def fill(s, e, out):
        z = splitmix64(seed, 2 * (e - s), 2 * s)
        u1 = ((z[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
        u2 = (z[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        r = np.sqrt(-2.0 * np.log(u1))
        out[s:e] = (r * np.cos(2.0 * math.pi * u2)).astype(np.float32)

    return _chunked(fill, n, np.float32)


def task_seed(rank: int, task: int) -> int:
    """Seed of task ``task`` of rank ``rank`` (rank*1000 + task)."""
    return rank * 1000 + task


def vadd_inputs(seed: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Operands a, b of a vector-add task: draws [0, n) and [n, 2n) of ``seed``."""
    return uniform_pm1(seed, n, 0), uniform_pm1(seed, n, n)


def vmul_inputs(seed: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Operands of a vector-multiply task: a in [-1, 1) from draws [0, n), and
    b = 1 + u/4 in [0.75, 1.25) from draws [n, 2n), so that up to 40 repeated
    products by b stay normal binary32 numbers (0.75**40 > 1e-5, 1.25**40 < 1e4)."""
    a = uniform_pm1(seed, n, 0)
    b = (np.float32(1.0) + uniform_pm1(seed, n, n) * np.float32(0.25)).astype(np.float32)
    return a, b


def sgemm_inputs(seed: int, m: int, n: int, k: int) -> tuple[np.ndarray, np.ndarray]:
    """Row-major A (m x k) from stream ``seed`` and B (k x n) from ``seed + 2**32``."""
    a = standard_normal(seed, m * k).reshape(m, k)
    b = standard_normal(seed + (1 << 32), k * n).reshape(k, n)
    return a, b


def sgemm_int_inputs(seed: int, m: int, n: int, k: int, lim: int = 16):
    """Integer-valued A, B with |x| <= lim: every product sum is exact in FP32."""
    za = splitmix64(seed, m * k) % np.uint64(2 * lim + 1)
    zb = splitmix64(seed + (1 << 32), k * n) % np.uint64(2 * lim + 1)
    a = (za.astype(np.int64) - lim).astype(np.float32).reshape(m, k)
    b = (zb.astype(np.int64) - lim).astype(np.float32).reshape(k, n)
    return a, b


# ---------------------------------------------------------------------------
# Workload recipes. A task spec names its type, sizes and seed; the operands
# are produced on demand by ``vadd_inputs`` / ``sgemm_inputs``.
# ---------------------------------------------------------------------------


@dataclass
class TaskSpec:
    rank: int
    index: int  # position in the rank's submission order
    kind: int  # TASK_VADD, TASK_SGEMM or TASK_VMUL
    n: int = 0  # vector length (VADD, VMUL) or N (SGEMM)
    m: int = 0
    k: int = 0  # K (SGEMM) or products per element (VMUL)
    seed: int = 0
    arrival_s: float = 0.0  # open-loop arrival time (serving workloads)

    @property
    def in_bytes(self) -> int:
        if self.kind in (TASK_VADD, TASK_VMUL):
            return 8 * self.n
        return 4 * (self.m * self.k + self.k * self.n)

    @property
    def out_bytes(self) -> int:
        if self.kind in (TASK_VADD, TASK_VMUL):
            return 4 * self.n
        return 4 * self.m * self.n

    @property
    def flops(self) -> int:
        if self.kind == TASK_VADD:
            return self.n
        if self.kind == TASK_VMUL:
            return self.n * self.k
        return 2 * self.m * self.n * self.k


@dataclass
class Workload:
    name: str
    ranks: int
    tasks: list[TaskSpec] = field(default_factory=list)

    def by_rank(self) -> list[list[TaskSpec]]:
        out: list[list[TaskSpec]] = [[] for _ in range(self.ranks)]
        for t in self.tasks:
            out[t.rank].append(t)
        for lst in out:
            lst.sort(key=lambda t: t.index)
        return out


def vadd_tiny(ranks: int = 4, per_rank: int = 8, n: int = 65536) -> Workload:
    """4 ranks x 8 vector adds of 65536 floats, seed rank*1000+task."""
    w = Workload(f"vadd_r{ranks}x{per_rank}_n{n}", ranks)
    for r in range(ranks):
        for t in range(per_rank):
            w.tasks.append(TaskSpec(r, t, TASK_VADD, n=n, seed=task_seed(r, t)))
    return w


def sgemm_square(ranks: int = 16, per_rank: int = 64, side: int = 512) -> Workload:
    """16 ranks x 64 SGEMM tasks, M=N=K=512, standard-normal operands."""
    w = Workload(f"sgemm_r{ranks}x{per_rank}_{side}cubed", ranks)
    for r in range(ranks):
        for t in range(per_rank):
            w.tasks.append(
                TaskSpec(r, t, TASK_SGEMM, n=side, m=side, k=side, seed=task_seed(r, t))
            )
    return w


def _draws(seed: int, n: int) -> np.ndarray:
    """Uniform float64 in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def serving_mix(
    ranks: int = 16,
    total: int = 4096,
    gap_us: float = 20.0,
    recipe_seed: int = 0x5E5E,
) -> Workload:
    """Poisson arrivals (mean gap per rank), 50/50 vector add and SGEMM.

    Vector-add length n = floor(2**(16 + 8u)); SGEMM square side uniform
    from {256, 512, 1024, 2048}. Exactly half of the tasks are of each type,
    in a seeded shuffle.
    """
    w = Workload(f"serving_r{ranks}_t{total}", ranks)
    per_rank = total // ranks
    kinds = np.array([TASK_VADD] * (total // 2) + [TASK_SGEMM] * (total - total // 2))
    order = np.argsort(_draws(recipe_seed, total), kind="stable")
    kinds = kinds[order]
    u = _draws(recipe_seed + 1, total)
    side_pick = (splitmix64(recipe_seed + 2, total) % np.uint64(4)).astype(np.int64)
    sides = np.array([256, 512, 1024, 2048])[side_pick]
    gaps = -np.log1p(-_draws(recipe_seed + 3, total)) * gap_us * 1e-6
    i = 0
    for r in range(ranks):
        t_arr = 0.0
        for t in range(per_rank):
            t_arr += float(gaps[i])
            if kinds[i] == TASK_VADD:
                n = int(math.floor(2.0 ** (16.0 + 8.0 * float(u[i]))))
                w.tasks.append(TaskSpec(r, t, TASK_VADD, n=n, seed=task_seed(r, t), arrival_s=t_arr))
            else:
                s = int(sides[i])
                w.tasks.append(
                    TaskSpec(r, t, TASK_SGEMM, n=s, m=s, k=s, seed=task_seed(r, t), arrival_s=t_arr)
                )
            i += 1
    return w


def grouped_mixed(ranks: int = 64, per_rank: int = 256, recipe_seed: int = 0xB47C) -> Workload:
    """SGEMM tasks with M, N, K drawn independently from {128, 192, ..., 2048}."""
    w = Workload(f"grouped_r{ranks}x{per_rank}", ranks)
    total = ranks * per_rank
    pick = (splitmix64(recipe_seed, 3 * total) % np.uint64(31)).astype(np.int64) * 64 + 128
    i = 0
    for r in range(ranks):
        for t in range(per_rank):
            m, n, k = (int(x) for x in pick[3 * i : 3 * i + 3])
            w.tasks.append(TaskSpec(r, t, TASK_SGEMM, n=n, m=m, k=k, seed=task_seed(r, t)))
            i += 1
    return w


def stress_mix(
    ranks: int = 128,
    per_rank: int = 8,
    vadd_median: float = 2.0 ** 20,
    side_median: float = 768.0,
    rate_per_rank_hz: float = 1000.0,
    recipe_seed: int = 0x57E5,
) -> Workload:
    """Open-loop stress mix: 70% vector add, 30% square SGEMM, Poisson
    arrivals. Vector-add length n = round(vadd_median * e^(1.5 Z)) clamped to
    [2^10, 2^28]; SGEMM side round(side_median * e^(0.7 Z)) clamped to
    [64, 4096] (Z standard normal). Smaller medians give the same shape mix
    at test size (the clamps then follow the medians' scale)."""
    w = Workload(f"stress_r{ranks}x{per_rank}", ranks)
    total = ranks * per_rank
    kind_u = _draws(recipe_seed, total)
    z = standard_normal(recipe_seed + 1, total)
    gaps = -np.log1p(-_draws(recipe_seed + 2, total)) / rate_per_rank_hz
    scale = vadd_median / 2.0 ** 20
    lo_n, hi_n = max(1, int(2 ** 10 * scale)), max(2, int(2 ** 28 * scale))
    sscale = side_median / 768.0
    lo_s, hi_s = max(1, int(64 * sscale)), max(2, int(4096 * sscale))
    i = 0
    for r in range(ranks):
        t_arr = 0.0
        for t in range(per_rank):
            t_arr += float(gaps[i])
            if kind_u[i] < 0.7:
                n = int(min(max(round(vadd_median * math.exp(1.5 * float(z[i]))), lo_n), hi_n))
                w.tasks.append(TaskSpec(r, t, TASK_VADD, n=n, seed=task_seed(r, t), arrival_s=t_arr))
            else:
                sd = int(min(max(round(side_median * math.exp(0.7 * float(z[i]))), lo_s), hi_s))
                w.tasks.append(TaskSpec(r, t, TASK_SGEMM, n=sd, m=sd, k=sd, seed=task_seed(r, t), arrival_s=t_arr))
            i += 1
    return w
