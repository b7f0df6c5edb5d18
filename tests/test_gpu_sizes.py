"""Parity at the full sizes of the measured workloads, in the launch
configuration the bench times.

* 4 ranks x 8 vector adds (n = 65536) and 16 ranks x 64 SGEMM 512^3: the
  bench's manager (ring of 64, per-rank slice of resident region + staging +
  64 MiB, ingest quantum 8, barrier mode), one step through the native SPMD
  harness with operands resident in HBM, then one with pinned host blocks
  (operands packed per rank at 256-byte multiples, so the manager merges the
  copies). Vector adds are compared bit for bit in full; SGEMM results on
  sampled rows and columns of every task (the oracle's dot products for those
  outputs), and the two legs must agree bit for bit.
* 64 ranks x 256 SGEMM with M, N, K from {128, ..., 2048}: the grouped
  launch as the bench runs it (one scheduler launch over 16384 tasks whose
  operands are leading blocks of per-rank 2048 x 2048 pools), sampled outputs
  of the first and last task of every rank and of four more per rank.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
import synth
from sgemm_bounds import SampledCheck, sample_indices

pytestmark = pytest.mark.gpu

SAMPLES = 8  # rows and columns sampled per SGEMM result


@pytest.fixture(scope="module")
def gvm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1511_07658_gb300 as g

    torch.cuda.set_device(0)
    return g


def al256(x):
    return (x + 255) // 256 * 256


def bits(x):
    return np.ascontiguousarray(x).view(np.uint32)


def operand_sizes(spec):
    if spec.kind == synth.TASK_VADD:
        return 4 * spec.n, 4 * spec.n, 4 * spec.n
    return 4 * spec.m * spec.k, 4 * spec.k * spec.n, 4 * spec.m * spec.n


def inputs_of(spec):
    if spec.kind == synth.TASK_VADD:
        return synth.vadd_inputs(spec.seed, spec.n)
    return synth.sgemm_inputs(spec.seed, spec.m, spec.n, spec.k)


_INPUTS = {}


def workload_inputs(w):
    """Every task's inputs, generated once per workload on all host cores."""
    if w.name not in _INPUTS:
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            got = list(ex.map(inputs_of, w.tasks))
        _INPUTS[w.name] = {(s.rank, s.index): x for s, x in zip(w.tasks, got)}
    return _INPUTS[w.name]


def run_bench_layout(g, w, path):
    """One resident step and one host-buffer step of workload w, laid out and
    launched as the bench does; returns, per task, its inputs and both C's."""
    R = w.ranks
    by_rank = w.by_rank()
    P = max(len(lst) for lst in by_rank)
    inputs = workload_inputs(w)
    res_off, res_need = {}, [0] * R
    in_off, in_need = {}, [0] * R
    out_off, out_need = {}, [0] * R
    for s in w.tasks:
        la, lb, lc = operand_sizes(s)
        o = res_need[s.rank]
        res_off[(s.rank, s.index)] = (o, o + la, o + la + lb)
        res_need[s.rank] = o + al256(la + lb + lc)
        in_off[(s.rank, s.index)] = in_need[s.rank]
        in_need[s.rank] += al256(la) + al256(lb)
        out_off[(s.rank, s.index)] = out_need[s.rank]
        out_need[s.rank] += al256(lc)
    resident = max(res_need)
    host_stage = max(sum(operand_sizes(s)) for s in w.tasks) * P
    slice_bytes = (resident + host_stage + (64 << 20) + (1 << 20) - 1) // (1 << 20) * (1 << 20)
    in_blocks = [torch.empty(max(x, 256), dtype=torch.uint8).pin_memory() for x in in_need]
    out_blocks = [torch.zeros(max(x, 256), dtype=torch.uint8).pin_memory() for x in out_need]

    def view(block, off, nbytes):
        return block[off : off + nbytes].view(torch.float32)

    with g.Manager(R, ring_depth=max(2, 1 << (P - 1).bit_length()), mode="barrier", sgemm_path=path,
                   slice_bytes=slice_bytes, resident_bytes=resident, ingest_quantum=8) as mgr:
        ranks = [mgr.attach(r) for r in range(R)]
        res_arrays, host_arrays = [], []
        for r in range(R):
            ra = (g.GvmTask * len(by_rank[r]))()
            ha = (g.GvmTask * len(by_rank[r]))()
            for i, s in enumerate(by_rank[r]):
                key = (s.rank, s.index)
                la, lb, lc = operand_sizes(s)
                a, b = inputs[key]
                ta = view(in_blocks[r], in_off[key], la)
                tb = view(in_blocks[r], in_off[key] + al256(la), lb)
                ta.copy_(torch.from_numpy(np.ascontiguousarray(a)).reshape(-1))
                tb.copy_(torch.from_numpy(np.ascontiguousarray(b)).reshape(-1))
                tc = view(out_blocks[r], out_off[key], lc)
                oa, ob, oc = res_off[key]
                ranks[r].write(oa, ta)
                ranks[r].write(ob, tb)
                for t in (ra[i], ha[i]):
                    t.type = g.GVM_TASK_VADD if s.kind == synth.TASK_VADD else g.GVM_TASK_SGEMM
                    t.m, t.n, t.k = s.m, s.n, s.k
                ra[i].flags = g.GVM_TASK_RESIDENT
                ra[i].a_off, ra[i].b_off, ra[i].c_off = oa, ob, oc
                ha[i].flags = 0
                ha[i].a, ha[i].b, ha[i].c = ta.data_ptr(), tb.data_ptr(), tc.data_ptr()
            res_arrays.append(ra)
            host_arrays.append(ha)
        torch.cuda.synchronize()
        mgr.spmd_run(ranks, res_arrays, 1)
        mgr.spmd_run(ranks, host_arrays, 1)
        assert mgr.stats()["device_status"] == 0
        out = {}
        for s in w.tasks:
            key = (s.rank, s.index)
            la, lb, lc = operand_sizes(s)
            shape = (s.n,) if s.kind == synth.TASK_VADD else (s.m, s.n)
            c_res = ranks[s.rank].resident_view(res_off[key][2], shape).cpu().numpy()
            c_host = view(out_blocks[s.rank], out_off[key], lc).numpy().reshape(shape).copy()
            out[key] = (inputs[key], c_res, c_host)
    return out


def test_vadd_4x8_bench_layout_bitexact(gvm):
    w = synth.vadd_tiny()
    out = run_bench_layout(gvm, w, "split3")
    assert len(out) == 32
    for s in w.tasks:
        (a, b), c_res, c_host = out[(s.rank, s.index)]
        ref = bits(oracle.vadd(a, b))
        assert np.array_equal(bits(c_res), ref), s
        assert np.array_equal(bits(c_host), ref), s


@pytest.mark.parametrize("path", ["split3", "split3_wide", "split3_tma", "fma"])
def test_sgemm512_16x64_bench_layout_sampled(gvm, path):
    w = synth.sgemm_square()
    out = run_bench_layout(gvm, w, path)
    assert len(out) == 1024
    rng = np.random.default_rng(1511)
    chk = SampledCheck()
    for s in w.tasks:
        (A, B), c_res, c_host = out[(s.rank, s.index)]
        assert np.array_equal(bits(c_res), bits(c_host)), f"{s}: resident and host legs differ"
        rows, cols = sample_indices(rng, s.m, SAMPLES), sample_indices(rng, s.n, SAMPLES)
        chk.add(c_host, A, B, rows, cols, label=str(s))
    assert chk.finish() < 1e-5


@pytest.mark.parametrize("path", ["split3", "split3_wide", "split3_tma"])
def test_grouped_64x256_sampled(gvm, path):
    # Every split3 tile form at the grouped benchmark's full size: the bench
    # runs whichever form the tuning table picks for this class.
    g = gvm
    R, P, side = 64, 256, 2048
    w = synth.grouped_mixed(ranks=R, per_rank=P)
    by_rank = w.by_rank()
    pool = 4 * side * side
    # Four distinct seeded pools (A then B), rank r holds pool r % 4.
    pools = [synth.standard_normal(synth.task_seed(p, 0), 2 * side * side) for p in range(4)]
    c_off, need = {}, [2 * pool] * R
    for s in w.tasks:
        c_off[(s.rank, s.index)] = need[s.rank]
        need[s.rank] += al256(4 * s.m * s.n)
    resident = max(need)
    rng = np.random.default_rng(7658)
    picks = []
    for r in range(R):
        more = rng.choice(np.arange(1, P - 1), 4, replace=False)
        picks += [(r, int(i)) for i in sorted({0, P - 1, *more.tolist()})]
    with g.Manager(R, ring_depth=max(2, 1 << (P - 1).bit_length()), mode="barrier", sgemm_path=path,
                   slice_bytes=resident + (4 << 20), resident_bytes=resident, ingest_quantum=8) as mgr:
        ranks = [mgr.attach(r) for r in range(R)]
        pinned = [torch.from_numpy(x).pin_memory() for x in pools]
        for r in range(R):
            ranks[r].write(0, pinned[r % 4])
        arrays = []
        for r in range(R):
            arr = (g.GvmTask * P)()
            for i, s in enumerate(by_rank[r]):
                t = arr[i]
                t.type, t.flags = g.GVM_TASK_SGEMM, g.GVM_TASK_RESIDENT
                t.m, t.n, t.k = s.m, s.n, s.k
                t.a_off, t.b_off, t.c_off = 0, pool, c_off[(r, s.index)]
            arrays.append(arr)
        torch.cuda.synchronize()
        mgr.spmd_run(ranks, arrays, 1)
        assert mgr.stats()["device_status"] == 0
        chk = SampledCheck()
        for r, i in picks:
            s = by_rank[r][i]
            src = pools[r % 4]
            A = src[: s.m * s.k].reshape(s.m, s.k)
            B = src[side * side : side * side + s.k * s.n].reshape(s.k, s.n)
            rows, cols = sample_indices(rng, s.m, SAMPLES), sample_indices(rng, s.n, SAMPLES)
            C = ranks[r].resident_view(c_off[(r, s.index)], (s.m, s.n))
            ri, ci = torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()
            chk.add_block(C[ri][:, ci].cpu().numpy(), A, B, rows, cols, label=str(s))
        assert chk.finish() < 1e-5
