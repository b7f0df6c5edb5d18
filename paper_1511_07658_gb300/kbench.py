"""Kernel-level timings of the task kernels alone (no manager).

    python -m paper_1511_07658_gb300.kbench            # all
    python -m paper_1511_07658_gb300.kbench 2048       # split3 SGEMM (both forms), one size
    python -m paper_1511_07658_gb300.kbench vadd       # vector add, 2^26 elements
    python -m paper_1511_07658_gb300.kbench link       # host-link copy rates

Times are CUDA events around repeated launches on the current stream, after
warm-up; inputs are device-resident random tensors. Used for the per-kernel
rooflines and as the small, self-contained cases the ncu captures run on.
"""
from __future__ import annotations

import sys

import torch

import paper_1511_07658_gb300 as g


def _time(fn, reps=10):
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


def sgemm(side: int, paths=("split3", "split3_fused", "split3_wide", "fma")) -> None:
    A = torch.randn(side, side, device="cuda")
    B = torch.randn(side, side, device="cuda")
    C = torch.empty(side, side, device="cuda")
    scratch = torch.empty(g.sgemm_scratch_bytes(side, side, side) + 256, dtype=torch.uint8, device="cuda")
    for path in paths:
        t = _time(lambda: g.sgemm_f32(A, B, C, path, scratch))
        print(f"sgemm {path} {side}^3: {t * 1e6:.1f} us {2 * side ** 3 / t / 1e12:.1f} TFLOP/s", flush=True)


def vadd(n: int, reps: int = 10) -> None:
    a = torch.randn(n, device="cuda")
    b = torch.randn(n, device="cuda")
    c = torch.empty(n, device="cuda")
    t = _time(lambda: g.vadd_f32(a, b, c), reps)
    print(f"vadd n={n}: {t * 1e6:.1f} us {12 * n / t / 1e9:.1f} GB/s", flush=True)


def link() -> None:
    n = 1 << 28
    h = torch.empty(n, dtype=torch.uint8).pin_memory()
    d = torch.empty(n, dtype=torch.uint8, device="cuda")
    t = _time(lambda: d.copy_(h, non_blocking=True))
    print(f"H2D 256 MiB: {n / t / 1e9:.1f} GB/s", flush=True)
    t = _time(lambda: h.copy_(d, non_blocking=True))
    print(f"D2H 256 MiB: {n / t / 1e9:.1f} GB/s", flush=True)
    hs = [torch.empty(n // 4, dtype=torch.uint8).pin_memory() for _ in range(4)]
    ds = [torch.empty(n // 4, dtype=torch.uint8, device="cuda") for _ in range(4)]
    ss = [torch.cuda.Stream() for _ in range(4)]

    def fan(duplex: bool):
        for i, (hh, dd, st) in enumerate(zip(hs, ds, ss)):
            with torch.cuda.stream(st):
                if duplex and i % 2:
                    hh.copy_(dd, non_blocking=True)
                else:
                    dd.copy_(hh, non_blocking=True)
        for st in ss:
            torch.cuda.current_stream().wait_stream(st)

    t = _time(lambda: fan(False))
    print(f"H2D 4 x 64 MiB on 4 streams: {n / t / 1e9:.1f} GB/s", flush=True)
    t = _time(lambda: fan(True))
    print(f"H2D + D2H 2 + 2 x 64 MiB: {n / t / 1e9:.1f} GB/s total", flush=True)
    # Many small copies, as the manager issues them: 16 streams (one per rank),
    # each copying 64 chunks; H2D alone, then with D2H of half the bytes on 16
    # more streams.
    for chunk in (1 << 20, 4 << 20):
        nch = 64
        hb = torch.empty(16 * nch * chunk, dtype=torch.uint8).pin_memory()
        db = torch.empty(16 * nch * chunk, dtype=torch.uint8, device="cuda")
        ho = torch.empty(16 * nch * chunk // 2, dtype=torch.uint8).pin_memory()
        do = torch.empty(16 * nch * chunk // 2, dtype=torch.uint8, device="cuda")
        sin = [torch.cuda.Stream() for _ in range(16)]
        sout = [torch.cuda.Stream() for _ in range(16)]

        def many(duplex: bool):
            for r in range(16):
                with torch.cuda.stream(sin[r]):
                    for i in range(nch):
                        o = (r * nch + i) * chunk
                        db[o:o + chunk].copy_(hb[o:o + chunk], non_blocking=True)
                if duplex:
                    with torch.cuda.stream(sout[r]):
                        for i in range(nch // 2):
                            o = (r * nch // 2 + i) * chunk
                            ho[o:o + chunk].copy_(do[o:o + chunk], non_blocking=True)
            for st in sin + (sout if duplex else []):
                torch.cuda.current_stream().wait_stream(st)

        byts = 16 * nch * chunk
        t = _time(lambda: many(False), reps=3)
        print(f"H2D 16 streams x 64 x {chunk >> 20} MiB: {byts / t / 1e9:.1f} GB/s", flush=True)
        t = _time(lambda: many(True), reps=3)
        print(f"H2D + D2H 16+16 streams, {chunk >> 20} MiB chunks: {1.5 * byts / t / 1e9:.1f} GB/s total", flush=True)


def main(argv) -> None:
    torch.cuda.set_device(0)
    what = argv[1] if len(argv) > 1 else "all"
    if what == "vadd":
        vadd(1 << 26, reps=3)
    elif what == "link":
        link()
    elif what.isdigit():
        sgemm(int(what), paths=("split3", "split3_fused", "split3_wide"))
    else:
        for side in (512, 2048, 4096):
            sgemm(side)
        vadd(1 << 28)
        link()


if __name__ == "__main__":
    main(sys.argv)
