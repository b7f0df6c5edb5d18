"""Parity of the shared-GPU manager against the CPU oracle, through the C ABI.

Each rank's tasks go through gvm_submit / gvm_flush / gvm_sync; every result
must equal the oracle's solo result for that task (vector add bit-exact,
SGEMM relative Frobenius error <= 1e-5), whatever else shares the GPU.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

from sgemm_bounds import check_sgemm  # noqa: E402


@pytest.fixture(scope="module")
def gvm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1511_07658_gb300 as g

    torch.cuda.set_device(0)
    return g


def bits(x):
    return np.ascontiguousarray(x).view(np.uint32)


def pinned(x):
    return torch.from_numpy(np.ascontiguousarray(x)).pin_memory()


def submit_spec(rk, spec):
    """Host-mode submission of a synth.TaskSpec; returns (seq, inputs, out)."""
    if spec.kind == synth.TASK_VADD:
        # The pinned inputs stay referenced until the task is synced (the
        # API's contract; the PS-1 / PS-2 modes copy them only at gvm_flush).
        a, b = synth.vadd_inputs(spec.seed, spec.n)
        out = torch.empty(spec.n, dtype=torch.float32).pin_memory()
        ta, tb = pinned(a), pinned(b)
        seq = rk.submit_vadd(ta, tb, out)
        return seq, (a, b, ta, tb), out
    if spec.kind == synth.TASK_VMUL:
        a, b = synth.vmul_inputs(spec.seed, spec.n)
        out = torch.empty(spec.n, dtype=torch.float32).pin_memory()
        ta, tb = pinned(a), pinned(b)
        seq = rk.submit_vmul(ta, tb, out, spec.k)
        return seq, (a, b, ta, tb), out
    A, B = synth.sgemm_inputs(spec.seed, spec.m, spec.n, spec.k)
    out = torch.empty(spec.m, spec.n, dtype=torch.float32).pin_memory()
    tA, tB = pinned(A), pinned(B)
    seq = rk.submit_sgemm(tA, tB, out)
    return seq, (A, B, tA, tB), out


def check_result(spec, inputs, out):
    if spec.kind == synth.TASK_VADD:
        assert np.array_equal(bits(out.numpy()), bits(oracle.vadd(inputs[0], inputs[1]))), spec
    elif spec.kind == synth.TASK_VMUL:
        assert np.array_equal(bits(out.numpy()), bits(oracle.vmul(inputs[0], inputs[1], spec.k))), spec
    else:
        try:
            check_sgemm(out.numpy(), inputs[0], inputs[1])
        except AssertionError as e:
            raise AssertionError(f"{spec}: {e}") from None


def run_workload(gvm, w, *, mode="barrier", path="split3", depth=16, slice_mb=128, direct=False):
    with gvm.Manager(w.ranks, ring_depth=depth, mode=mode, sgemm_path=path, slice_bytes=slice_mb << 20,
                     direct_output=direct) as mgr:
        ranks = [mgr.attach(r) for r in range(w.ranks)]
        jobs = []
        for spec in w.tasks:
            jobs.append((spec, *submit_spec(ranks[spec.rank], spec)))
        mgr.flush()
        for spec, seq, inputs, out in jobs:
            ranks[spec.rank].sync(seq)
        stats = mgr.stats()
        results = {(s.rank, s.index): out for s, _, _, out in jobs}
        for spec, seq, inputs, out in jobs:
            check_result(spec, inputs, out)
    assert stats["device_status"] == 0
    return results


@pytest.mark.parametrize("mode", ["barrier", "continuous"])
def test_vadd_tiny_config_bitexact(gvm, mode):
    """4 ranks x 8 vector adds, n = 65536, seed rank*1000 + task."""
    run_workload(gvm, synth.vadd_tiny(), mode=mode)


@pytest.mark.parametrize("path", ["fma", "split3", "split3_wide", "split3_tma"])
def test_sgemm_shared_subset(gvm, path):
    """16 ranks sharing the GPU, SGEMM 512^3 (two tasks per rank here; the
    full 64-per-rank configuration runs in test_gpu_sizes)."""
    run_workload(gvm, synth.sgemm_square(ranks=16, per_rank=2), path=path, slice_mb=64)


@pytest.mark.parametrize("path", ["fma", "split3", "split3_wide", "split3_tma"])
def test_mixed_ragged_tasks(gvm, path):
    w = synth.Workload("mixed", 3)
    shapes = [(1, 1, 1), (64, 64, 64), (130, 257, 65), (5, 300, 17)]
    i = 0
    for r in range(3):
        for t in range(6):
            if (r + t) % 2 == 0:
                w.tasks.append(synth.TaskSpec(r, t, synth.TASK_VADD, n=[0, 1, 4099, 70001][i % 4], seed=1000 + i))
            else:
                m, n, k = shapes[i % 4]
                w.tasks.append(synth.TaskSpec(r, t, synth.TASK_SGEMM, m=m, n=n, k=k, seed=2000 + i))
            i += 1
    run_workload(gvm, w, path=path, depth=8)


@pytest.mark.parametrize("mode", ["barrier", "continuous"])
@pytest.mark.parametrize("path", ["fma", "split3", "split3_wide", "split3_tma"])
def test_vmul_tasks_in_mix(gvm, mode, path):
    """Vector-multiply tasks (the paper's VecMult, 15 products) shared with
    vector adds and matrix multiplies, ragged lengths, host mode."""
    w = synth.Workload("vmul-mix", 4)
    i = 0
    for r in range(4):
        for t in range(5):
            kind = (r + t) % 3
            if kind == 0:
                w.tasks.append(synth.TaskSpec(r, t, synth.TASK_VMUL, n=[0, 3, 70001, 1 << 20][i % 4], k=[15, 1, 15, 40][i % 4], seed=3000 + i))
            elif kind == 1:
                w.tasks.append(synth.TaskSpec(r, t, synth.TASK_VADD, n=33333 + i, seed=4000 + i))
            else:
                w.tasks.append(synth.TaskSpec(r, t, synth.TASK_SGEMM, m=130, n=257, k=65, seed=5000 + i))
            i += 1
    run_workload(gvm, w, mode=mode, path=path, depth=8)


def test_vmul_resident_and_bad_iters(gvm):
    n = 50001
    a, b = synth.vmul_inputs(synth.task_seed(1, 2), n)
    with gvm.Manager(1, ring_depth=4, slice_bytes=16 << 20, resident_bytes=12 * 65536) as mgr:
        rk = mgr.attach(0)
        rk.write(0, torch.from_numpy(a))
        rk.write(4 * 65536, torch.from_numpy(b))
        seq = rk.submit_vmul_resident(0, 4 * 65536, 8 * 65536, n, 15)
        mgr.flush()
        rk.sync(seq)
        c = torch.empty(n)
        rk.read(8 * 65536, c)
        assert np.array_equal(bits(c.numpy()), bits(oracle.vmul(a, b, 15)))
        for iters in (0, 1025):
            with pytest.raises(RuntimeError):
                rk.submit_vmul_resident(0, 4 * 65536, 8 * 65536, n, iters)
        assert mgr.stats()["device_status"] == 0


def _ps_mix():
    w = synth.Workload("ps-mix", 5)
    shapes = [(1, 1, 1), (130, 257, 65), (512, 512, 512), (5, 300, 17)]
    i = 0
    for r in range(5):
        for t in range(6):
            kind = (r + 2 * t) % 3
            if kind == 0:
                w.tasks.append(synth.TaskSpec(r, t, synth.TASK_VADD, n=[0, 7, 70001, 1 << 20][i % 4], seed=6000 + i))
            elif kind == 1:
                w.tasks.append(synth.TaskSpec(r, t, synth.TASK_VMUL, n=[1, 4099, 65536, 300001][i % 4], k=15, seed=7000 + i))
            else:
                m, n, k = shapes[i % 4]
                w.tasks.append(synth.TaskSpec(r, t, synth.TASK_SGEMM, m=m, n=n, k=k, seed=8000 + i))
            i += 1
    return w


@pytest.mark.parametrize("mode", ["ps1", "ps2"])
@pytest.mark.parametrize("path", ["fma", "split3", "split3_wide", "split3_tma"])
def test_paper_stream_modes(gvm, mode, path):
    """PS-1 / PS-2 (the host issues each task's copies and kernel at the
    request barrier): oracle parity, and bitwise the same results as the
    persistent scheduler on the same workload."""
    w = _ps_mix()
    ps = run_workload(gvm, w, mode=mode, path=path, depth=8)
    sched = run_workload(gvm, w, mode="barrier", path=path, depth=8)
    for key in ps:
        assert np.array_equal(bits(ps[key].numpy()), bits(sched[key].numpy())), key


@pytest.mark.parametrize("mode", ["barrier", "continuous"])
@pytest.mark.parametrize("path", ["fma", "split3"])
def test_direct_output(gvm, mode, path):
    """Results written by the scheduler straight into the page-locked host
    buffers (no output staging, no copy): oracle parity, bitwise the same as
    the staged path, and no staging held for outputs."""
    w = _ps_mix()
    direct = run_workload(gvm, w, mode=mode, path=path, depth=8, direct=True)
    staged = run_workload(gvm, w, mode=mode, path=path, depth=8, direct=False)
    for key in direct:
        assert np.array_equal(bits(direct[key].numpy()), bits(staged[key].numpy())), key


def test_direct_output_takes_no_output_staging(gvm):
    n = 1 << 20
    a, b = synth.vadd_inputs(5, n)
    ta, tb = pinned(a), pinned(b)
    for direct, want in ((True, 8 * n), (False, 12 * n)):
        out = torch.empty(n).pin_memory()
        with gvm.Manager(1, ring_depth=4, slice_bytes=64 << 20, direct_output=direct) as mgr:
            rk = mgr.attach(0)
            seq = rk.submit_vadd(ta, tb, out)
            assert mgr.stats()["staged_bytes"] == want
            mgr.flush()
            rk.sync(seq)
        assert np.array_equal(bits(out.numpy()), bits(oracle.vadd(a, b)))


@pytest.mark.parametrize("mode", ["barrier", "continuous", "ps1"])
def test_pageable_host_buffers(gvm, mode):
    """Host-mode tasks on pageable (not page-locked) buffers, alone and mixed
    with page-locked ones: results equal the oracle's."""
    specs = [("vadd", 70001), ("vmul", 4099), ("sgemm", (130, 257, 65)), ("sgemm", (256, 256, 256))]
    with gvm.Manager(2, ring_depth=8, mode=mode, sgemm_path="split3", slice_bytes=32 << 20) as mgr:
        ranks = [mgr.attach(r) for r in range(2)]
        jobs = []
        for r, rk in enumerate(ranks):
            for i, (kind, shape) in enumerate(specs):
                pin = (r + i) % 2 == 0  # half page-locked, half pageable
                mk = (lambda x: torch.from_numpy(np.ascontiguousarray(x)).pin_memory()) if pin else \
                     (lambda x: torch.from_numpy(np.ascontiguousarray(x)).clone())
                seed = synth.task_seed(r, 50 + i)
                if kind == "sgemm":
                    m, n, k = shape
                    A, B = synth.sgemm_inputs(seed, m, n, k)
                    ta, tb = mk(A), mk(B)
                    out = torch.full((m, n), float("nan"))
                    out = out.pin_memory() if pin else out
                    seq = rk.submit_sgemm(ta, tb, out)
                    spec = synth.TaskSpec(r, i, synth.TASK_SGEMM, m=m, n=n, k=k)
                    jobs.append((rk, seq, spec, (A, B, ta, tb), out))
                else:
                    n = shape
                    a, b = synth.vmul_inputs(seed, n) if kind == "vmul" else synth.vadd_inputs(seed, n)
                    ta, tb = mk(a), mk(b)
                    out = torch.full((n,), float("nan"))
                    out = out.pin_memory() if pin else out
                    if kind == "vmul":
                        seq = rk.submit_vmul(ta, tb, out, 15)
                        spec = synth.TaskSpec(r, i, synth.TASK_VMUL, n=n, k=15)
                    else:
                        seq = rk.submit_vadd(ta, tb, out)
                        spec = synth.TaskSpec(r, i, synth.TASK_VADD, n=n)
                    jobs.append((rk, seq, spec, (a, b, ta, tb), out))
        mgr.flush_if_barrier()
        for rk, seq, spec, inputs, out in jobs:
            rk.sync(seq)
            check_result(spec, inputs, out)
        assert mgr.stats()["device_status"] == 0


@pytest.mark.parametrize("mode", ["ps1", "ps2"])
def test_paper_stream_modes_barrier_rules(gvm, mode):
    """A task submitted after the last gvm_flush does not run: gvm_sync says
    GVM_ESTATE until the next flush; shutdown issues what is still pending."""
    n = 4096
    a, b = synth.vadd_inputs(11, n)
    with gvm.Manager(2, ring_depth=4, mode=mode, slice_bytes=8 << 20) as mgr:
        rk = mgr.attach(0)
        out = torch.empty(n).pin_memory()
        ta, tb = pinned(a), pinned(b)  # referenced until synced
        seq = rk.submit_vadd(ta, tb, out)
        with pytest.raises(RuntimeError):
            rk.sync(seq)
        mgr.flush()
        rk.sync(seq)
        assert np.array_equal(bits(out.numpy()), bits(oracle.vadd(a, b)))
        out2 = torch.empty(n).pin_memory()
        rk.submit_vmul(ta, tb, out2, 15)
        st = mgr.stats()
        assert st["launches"] == 1 and st["h2d_bytes"] == 8 * n and st["d2h_bytes"] == 4 * n
    assert np.array_equal(bits(out2.numpy()), bits(oracle.vmul(a, b, 15)))


@pytest.mark.parametrize("path", ["fma", "split3", "split3_wide", "split3_tma"])
def test_solo_equals_mix_bitwise(gvm, path):
    """A task's result alone on the GPU equals its result in the mix, bit for
    bit (the tile shape is a function of the task's shape only)."""
    w = synth.Workload("mix", 4)
    for r in range(4):
        for t in range(3):
            if t == 1:
                w.tasks.append(synth.TaskSpec(r, t, synth.TASK_VADD, n=50000 + r, seed=synth.task_seed(r, t)))
            else:
                w.tasks.append(
                    synth.TaskSpec(r, t, synth.TASK_SGEMM, m=192 + 64 * r, n=320, k=256, seed=synth.task_seed(r, t))
                )
    mixed = run_workload(gvm, w, path=path)
    for spec in w.tasks:
        solo = synth.Workload("solo", 4, [spec])
        alone = run_workload(gvm, solo, path=path)
        key = (spec.rank, spec.index)
        assert np.array_equal(bits(alone[key].numpy()), bits(mixed[key].numpy())), spec


def test_resident_mode(gvm):
    """Inputs placed in the rank's resident region; no copies in the task."""
    m = n = k = 256
    nv = 10000
    res = 4 * (m * k + k * n + m * n) + 3 * 4 * nv + 1024
    with gvm.Manager(2, ring_depth=8, sgemm_path="split3", slice_bytes=32 << 20, resident_bytes=res) as mgr:
        for r in range(2):
            rk = mgr.attach(r)
            A, B = synth.sgemm_inputs(synth.task_seed(r, 0), m, n, k)
            a, b = synth.vadd_inputs(synth.task_seed(r, 1), nv)
            offA, offB, offC = 0, 4 * m * k, 4 * (m * k + k * n)
            offa = 4 * (m * k + k * n + m * n)
            offb, offc = offa + 4 * nv, offa + 8 * nv
            rk.write(offA, torch.from_numpy(A))
            rk.write(offB, torch.from_numpy(B))
            rk.write(offa, torch.from_numpy(a))
            rk.write(offb, torch.from_numpy(b))
            s0 = rk.submit_sgemm_resident(offA, offB, offC, m, n, k)
            s1 = rk.submit_vadd_resident(offa, offb, offc, nv)
            mgr.flush()
            rk.sync(s1)
            assert rk.poll(s0)
            C = torch.empty(m, n)
            c = torch.empty(nv)
            rk.read(offC, C)
            rk.read(offc, c)
            check_sgemm(C.numpy(), A, B)
            assert np.array_equal(bits(c.numpy()), bits(oracle.vadd(a, b)))


def test_rank_isolation_canaries(gvm):
    """Data of different ranks coexist safely (Section 5): tasks touch only
    their own rank's buffers, so canaries elsewhere in the arena survive."""
    R = 4
    nv = 4096
    res = 1 << 20
    with gvm.Manager(R, ring_depth=8, sgemm_path="split3", slice_bytes=16 << 20, resident_bytes=res) as mgr:
        ranks = [mgr.attach(r) for r in range(R)]
        canary = torch.full((res // 4,), 1234.5)
        for rk in ranks:
            rk.write(0, canary)
        seqs = []
        for r, rk in enumerate(ranks):
            a, b = synth.vadd_inputs(r, nv)
            rk.write(0, torch.from_numpy(a))
            rk.write(4 * nv, torch.from_numpy(b))
            seqs.append(rk.submit_vadd_resident(0, 4 * nv, 8 * nv, nv))
            A, B = synth.sgemm_inputs(r + 50, 64, 64, 64)
            base = 16 * nv
            rk.write(base, torch.from_numpy(A))
            rk.write(base + 4 * 64 * 64, torch.from_numpy(B))
            seqs.append(rk.submit_sgemm_resident(base, base + 4 * 4096, base + 8 * 4096, 64, 64, 64))
        mgr.flush()
        for r, rk in enumerate(ranks):
            rk.sync(seqs[2 * r + 1])
            back = torch.empty(res // 4)
            rk.read(0, back)
            tail = back[(16 * nv + 12 * 4096) // 4 :]
            assert torch.all(tail == 1234.5), f"rank {r} canary overwritten"
            assert torch.all(back[3 * nv : 4 * nv] == 1234.5)


def test_errors_and_backpressure(gvm):
    import ctypes

    with gvm.Manager(1, ring_depth=4, sgemm_path="fma", slice_bytes=8 << 20) as mgr:
        rk = mgr.attach(0)
        with pytest.raises(gvm.GvmError) as e:
            mgr.attach(0)
        assert e.value.code == gvm.GVM_EBUSY
        # device memory may not be named by a host-mode task
        a = torch.zeros(16, device="cuda")
        with pytest.raises(gvm.GvmError) as e:
            rk.submit_vadd(a, a, a)
        assert e.value.code == gvm.GVM_EINVAL
        # bad shapes
        t = gvm.GvmTask()
        t.type, t.m, t.n, t.k = gvm.GVM_TASK_SGEMM, 0, 4, 4
        assert gvm.lib().gvm_submit(rk.handle, ctypes.byref(t), None) == gvm.GVM_EINVAL
        t.type = 7
        assert gvm.lib().gvm_submit(rk.handle, ctypes.byref(t), None) == gvm.GVM_EINVAL
        # resident offsets outside the (empty) resident region
        with pytest.raises(gvm.GvmError) as e:
            rk.submit_vadd_resident(0, 0, 0, 16)
        assert e.value.code == gvm.GVM_EINVAL
        # too big for the staging ring ever
        big = torch.empty(3 << 20).pin_memory()
        with pytest.raises(gvm.GvmError) as e:
            rk.submit_vadd(big, big, big, block=False)
        assert e.value.code == gvm.GVM_ENOMEM
        # ring full: 4 slots, nothing runs until flush (barrier mode)
        x = torch.ones(1000).pin_memory()
        outs = [torch.empty(1000).pin_memory() for _ in range(5)]
        seqs = [rk.submit_vadd(x, x, outs[i], block=False) for i in range(4)]
        with pytest.raises(gvm.GvmError) as e:
            rk.submit_vadd(x, x, outs[4], block=False)
        assert e.value.code == gvm.GVM_EAGAIN
        mgr.flush()
        rk.sync(seqs[-1])
        seqs.append(rk.submit_vadd(x, x, outs[4], block=False))
        mgr.flush()
        rk.sync(seqs[-1])
        for o in outs:
            assert torch.all(o == 2.0)


def test_order_and_times(gvm):
    """Per rank, sync(seq) implies every earlier task of the rank is done,
    and device timestamps are consistent."""
    w = synth.vadd_tiny(ranks=2, per_rank=6, n=30000)
    with gvm.Manager(2, ring_depth=8, mode="continuous") as mgr:
        ranks = [mgr.attach(r) for r in range(2)]
        jobs = [(spec, *submit_spec(ranks[spec.rank], spec)) for spec in w.tasks]
        last = {}
        for spec, seq, inputs, out in jobs:
            last[spec.rank] = seq
        for r, rk in enumerate(ranks):
            rk.sync(last[r])
            for spec, seq, inputs, out in jobs:
                if spec.rank == r:
                    assert rk.poll(seq)
                    t0, t1 = rk.task_times(seq)
                    assert 0 < t0 <= t1
                    check_result(spec, inputs, out)


@pytest.mark.parametrize("mode", ["barrier", "continuous", "ps1", "ps2"])
def test_spmd_harness_steps(gvm, mode):
    # gvm_spmd_run: one native thread per rank submits its batch each step,
    # flush (barrier mode), sync. Every step's results must be the oracle's;
    # the last step's outputs are checked (each step rewrites them), and the
    # per-step times must be positive.
    w = synth.Workload(name="spmd", ranks=4, tasks=[
        synth.TaskSpec(rank=r, index=i, kind=synth.TASK_VADD if i % 2 == 0 else synth.TASK_SGEMM,
                       seed=synth.task_seed(r, i), n=65536 + 257 * r if i % 2 == 0 else 300,
                       m=0 if i % 2 == 0 else 130 + r, k=0 if i % 2 == 0 else 96)
        for r in range(4) for i in range(6)])
    with gvm.Manager(w.ranks, ring_depth=8, mode=mode, sgemm_path="split3", slice_bytes=64 << 20) as mgr:
        ranks = [mgr.attach(r) for r in range(w.ranks)]
        arrays = [(gvm.GvmTask * 6)() for _ in range(w.ranks)]
        keep = []
        for spec in w.tasks:
            t = arrays[spec.rank][spec.index]
            if spec.kind == synth.TASK_VADD:
                a, b = synth.vadd_inputs(spec.seed, spec.n)
                ins = (pinned(a), pinned(b))
                out = torch.empty(spec.n, dtype=torch.float32).pin_memory()
                t.type, t.n = gvm.GVM_TASK_VADD, spec.n
                ref = (a, b)
            else:
                A, B = synth.sgemm_inputs(spec.seed, spec.m, spec.n, spec.k)
                ins = (pinned(A), pinned(B))
                out = torch.empty(spec.m, spec.n, dtype=torch.float32).pin_memory()
                t.type, t.m, t.n, t.k = gvm.GVM_TASK_SGEMM, spec.m, spec.n, spec.k
                ref = (A, B)
            t.flags = 0
            t.a, t.b, t.c = ins[0].data_ptr(), ins[1].data_ptr(), out.data_ptr()
            keep.append((spec, ins, out, ref))
        if mode != "continuous":
            dev, launch, host, lat = mgr.spmd_run(ranks, arrays, 3, latency=True)
            assert all(x > 0 for x in dev)
            if mode == "barrier":
                assert all(x > 0 for x in launch)
                assert all(l <= d for l, d in zip(launch, dev))
            # host-clock latency of every task: positive, in submission order
            # within a step (collected in order), never longer than its step
            for r in range(w.ranks):
                assert len(lat[r]) == 3 * 6
                for i in range(3):
                    step = lat[r][6 * i:6 * i + 6]
                    assert all(x > 0 for x in step)
                    assert step == sorted(step)
                    assert step[-1] * 1e3 <= host[i] + 1e-6
        else:
            n = len(ranks)
            import ctypes

            hs = (ctypes.c_void_p * n)(*[r.handle for r in ranks])
            tp = (ctypes.POINTER(gvm.GvmTask) * n)(*[ctypes.cast(a, ctypes.POINTER(gvm.GvmTask)) for a in arrays])
            cnt = (ctypes.c_uint32 * n)(*[6] * n)
            host = (ctypes.c_double * 3)()
            rc = gvm._abi.lib().gvm_spmd_run(mgr.handle, hs, tp, cnt, n, 3, None, None, host, None)
            assert rc == 0, rc
            host = list(host)
        assert all(x > 0 for x in host)
        for spec, _, out, ref in keep:
            check_result(spec, ref, out)
        assert mgr.stats()["device_status"] == 0


@pytest.mark.parametrize("mode", ["barrier", "ps1"])
def test_spmd_overlapped_steps(gvm, mode):
    """gvm_spmd_run_overlapped: step i + 1 is submitted and flushed before
    step i is collected; even and odd steps write separate host outputs, and
    both hold the oracle's results afterwards."""
    R, per = 4, 5
    specs = []
    for r in range(R):
        for i in range(per):
            if i % 2 == 0:
                specs.append(synth.TaskSpec(r, i, synth.TASK_SGEMM, m=130 + r, n=200, k=96, seed=synth.task_seed(r, i)))
            else:
                specs.append(synth.TaskSpec(r, i, synth.TASK_VMUL, n=30001 + r, k=15, seed=synth.task_seed(r, i)))
    with gvm.Manager(R, ring_depth=16, mode=mode, sgemm_path="split3", slice_bytes=32 << 20) as mgr:
        ranks = [mgr.attach(r) for r in range(R)]
        even = [(gvm.GvmTask * per)() for _ in range(R)]
        odd = [(gvm.GvmTask * per)() for _ in range(R)]
        keep = []
        for spec in specs:
            if spec.kind == synth.TASK_SGEMM:
                A, B = synth.sgemm_inputs(spec.seed, spec.m, spec.n, spec.k)
                ins, shape = (pinned(A), pinned(B)), (spec.m, spec.n)
            else:
                a, b = synth.vmul_inputs(spec.seed, spec.n)
                ins, shape = (pinned(a), pinned(b)), (spec.n,)
            outs = (torch.full(shape, float("nan")).pin_memory(), torch.full(shape, float("nan")).pin_memory())
            for arr, out in ((even, outs[0]), (odd, outs[1])):
                t = arr[spec.rank][spec.index]
                t.type = gvm.GVM_TASK_SGEMM if spec.kind == synth.TASK_SGEMM else gvm.GVM_TASK_VMUL
                t.flags = 0
                t.m, t.n, t.k = spec.m, spec.n, spec.k
                t.a, t.b, t.c = ins[0].data_ptr(), ins[1].data_ptr(), out.data_ptr()
            keep.append((spec, ins, outs))
        total, done = mgr.spmd_run_overlapped(ranks, even, odd, 5)
        assert total > 0 and len(done) == 5 and all(x > 0 for x in done)
        assert done == sorted(done) and done[-1] <= total
        assert mgr.stats()["device_status"] == 0
    for spec, ins, outs in keep:
        for out in outs:
            check_result(spec, (ins[0].numpy(), ins[1].numpy()), out)


@pytest.mark.parametrize("nphases,in_streams", [(1, 0), (3, 0), (3, 1)])
def test_spmd_pipelined_steps(gvm, nphases, in_streams):
    """gvm_spmd_run_pipelined: with nphases steps in flight, step i uses phase
    i % nphases and is collected after step i + nphases - 1 is submitted;
    every phase's host outputs hold the oracle's results afterwards (7 steps:
    each phase runs at least twice, the last ones collected after the final
    submit). in_streams = 1: every rank's input copies share one stream
    (gvm_config.copy_in_streams)."""
    R, per, steps = 3, 4, 7
    specs = []
    for r in range(R):
        for i in range(per):
            if i % 2 == 0:
                specs.append(synth.TaskSpec(r, i, synth.TASK_SGEMM, m=100 + r, n=260, k=64, seed=synth.task_seed(r, i)))
            else:
                specs.append(synth.TaskSpec(r, i, synth.TASK_VADD, n=40003 + r, seed=synth.task_seed(r, i)))
    with gvm.Manager(R, ring_depth=16, mode="barrier", sgemm_path="split3", slice_bytes=32 << 20,
                     copy_in_streams=in_streams) as mgr:
        ranks = [mgr.attach(r) for r in range(R)]
        phases = [[(gvm.GvmTask * per)() for _ in range(R)] for _ in range(nphases)]
        keep = []
        for spec in specs:
            if spec.kind == synth.TASK_SGEMM:
                A, B = synth.sgemm_inputs(spec.seed, spec.m, spec.n, spec.k)
                ins, shape = (pinned(A), pinned(B)), (spec.m, spec.n)
            else:
                a, b = synth.vadd_inputs(spec.seed, spec.n)
                ins, shape = (pinned(a), pinned(b)), (spec.n,)
            outs = [torch.full(shape, float("nan")).pin_memory() for _ in range(nphases)]
            for arr, out in zip(phases, outs):
                t = arr[spec.rank][spec.index]
                t.type = gvm.GVM_TASK_SGEMM if spec.kind == synth.TASK_SGEMM else gvm.GVM_TASK_VADD
                t.flags = 0
                t.m, t.n, t.k = spec.m, spec.n, spec.k
                t.a, t.b, t.c = ins[0].data_ptr(), ins[1].data_ptr(), out.data_ptr()
            keep.append((spec, ins, outs))
        total, done = mgr.spmd_run_pipelined(ranks, phases, steps)
        assert total > 0 and len(done) == steps and all(x > 0 for x in done)
        assert done == sorted(done) and done[-1] <= total
        assert mgr.stats()["device_status"] == 0
    for spec, ins, outs in keep:
        for out in outs:
            check_result(spec, (ins[0].numpy(), ins[1].numpy()), out)


@pytest.mark.parametrize("max_inflight", [1, 3])
def test_open_loop_harness(gvm, max_inflight):
    """gvm_open_loop_run (continuous mode): paced arrivals, at most
    max_inflight tasks per rank outstanding; every result equals the
    oracle's, every latency is non-negative, the span covers the arrivals."""
    R, per = 4, 6
    w = synth.stress_mix(ranks=R, per_rank=per, vadd_median=4096, side_median=96, rate_per_rank_hz=5000.0)
    with gvm.Manager(R, ring_depth=8, mode="continuous", sgemm_path="split3", slice_bytes=16 << 20) as mgr:
        ranks = [mgr.attach(r) for r in range(R)]
        by_rank = w.by_rank()
        arrays, arrivals, keep = [], [], []
        for r in range(R):
            arr = (gvm.GvmTask * per)()
            for i, spec in enumerate(by_rank[r]):
                t = arr[i]
                seq, inputs, out = None, None, None
                if spec.kind == synth.TASK_VADD:
                    a, b = synth.vadd_inputs(spec.seed, spec.n)
                    ins = (pinned(a), pinned(b))
                    out = torch.full((spec.n,), float("nan")).pin_memory()
                    t.type, t.n = gvm.GVM_TASK_VADD, spec.n
                    inputs = (a, b)
                else:
                    A, B = synth.sgemm_inputs(spec.seed, spec.m, spec.n, spec.k)
                    ins = (pinned(A), pinned(B))
                    out = torch.full((spec.m, spec.n), float("nan")).pin_memory()
                    t.type, t.m, t.n, t.k = gvm.GVM_TASK_SGEMM, spec.m, spec.n, spec.k
                    inputs = (A, B)
                t.flags = 0
                t.a, t.b, t.c = ins[0].data_ptr(), ins[1].data_ptr(), out.data_ptr()
                keep.append((spec, inputs, ins, out))
            arrays.append(arr)
            arrivals.append([int(s.arrival_s * 1e9) for s in by_rank[r]])
        span, lat = mgr.open_loop_run(ranks, arrays, arrivals, max_inflight=max_inflight)
        assert span >= max(max(a) for a in arrivals) / 1e9
        assert all(len(l) == per and all(x >= 0 for x in l) for l in lat)
        assert mgr.stats()["device_status"] == 0
    for spec, inputs, ins, out in keep:
        check_result(spec, inputs, out)


@pytest.mark.parametrize("slice_mb", [64, 2])
def test_batch_from_contiguous_host_blocks(gvm, slice_mb):
    # A rank's operands in one pinned block (A then B per task) and its
    # outputs in another: gvm_submit_many packs the batch's staging the same
    # way and merges adjacent copies. Sizes mix 256-byte multiples (merged)
    # with others (not merged). With a 2 MiB slice the batch is admitted a
    # prefix at a time (the binding flushes and syncs in between).
    specs = []
    for i in range(10):
        if i % 3 == 0:
            specs.append(("v", 65536 if i % 2 == 0 else 1000 + i))
        else:
            specs.append(("g", (128, 256, 64) if i % 2 == 0 else (67, 130, 45)))
    R = 2
    with gvm.Manager(R, ring_depth=16, sgemm_path="split3", slice_bytes=slice_mb << 20) as mgr:
        ranks = [mgr.attach(r) for r in range(R)]
        checks = []
        arrays = []
        for r in range(R):
            sizes = []
            for kind, shp in specs:
                if kind == "v":
                    sizes.append((4 * shp, 4 * shp, 4 * shp))
                else:
                    m, n, k = shp
                    sizes.append((4 * m * k, 4 * k * n, 4 * m * n))
            al = lambda x: (x + 255) // 256 * 256  # noqa: E731
            inb = torch.zeros(sum(al(a) + al(b) for a, b, _ in sizes), dtype=torch.uint8).pin_memory()
            outb = torch.zeros(sum(al(c) for _, _, c in sizes), dtype=torch.uint8).pin_memory()
            arr = (gvm.GvmTask * len(specs))()
            io = oo = 0
            for i, ((kind, shp), (la, lb, lc)) in enumerate(zip(specs, sizes)):
                ta = inb[io:io + la].view(torch.float32)
                tb = inb[io + al(la):io + al(la) + lb].view(torch.float32)
                tc = outb[oo:oo + lc].view(torch.float32)
                io += al(la) + al(lb)
                oo += al(lc)
                seed = synth.task_seed(r, i)
                t = arr[i]
                if kind == "v":
                    a, b = synth.vadd_inputs(seed, shp)
                    t.type, t.n = gvm.GVM_TASK_VADD, shp
                    checks.append((synth.TaskSpec(rank=r, index=i, kind=synth.TASK_VADD, n=shp), (a, b), tc))
                else:
                    m, n, k = shp
                    a, b = synth.sgemm_inputs(seed, m, n, k)
                    t.type, t.m, t.n, t.k = gvm.GVM_TASK_SGEMM, m, n, k
                    checks.append((synth.TaskSpec(rank=r, index=i, kind=synth.TASK_SGEMM, m=m, n=n, k=k), (a, b),
                                   tc.view(m, n)))
                ta.copy_(torch.from_numpy(np.ascontiguousarray(a)).reshape(-1))
                tb.copy_(torch.from_numpy(np.ascontiguousarray(b)).reshape(-1))
                t.flags = 0
                t.a, t.b, t.c = ta.data_ptr(), tb.data_ptr(), tc.data_ptr()
            arrays.append((arr, inb, outb))
        lasts = []
        for r in range(R):
            first, cnt = ranks[r].submit_many(arrays[r][0])
            assert cnt == len(specs)
            lasts.append(first + cnt - 1)
        mgr.flush()
        for r in range(R):
            ranks[r].sync(lasts[r])
        for spec, ins, out in checks:
            check_result(spec, ins, out)
        assert mgr.stats()["device_status"] == 0


@pytest.mark.parametrize("mode,path", [("barrier", "split3"), ("continuous", "split3"), ("barrier", "fma"),
                                       ("barrier", "split3_wide"), ("continuous", "split3_wide"),
                                       ("barrier", "split3_tma"), ("continuous", "split3_tma")])
def test_stress_mix_ragged_sizes(gvm, mode, path):
    # The stress config's shape mix (70% vector adds with lognormal lengths,
    # 30% square SGEMMs with lognormal sides; most sizes odd, none aligned)
    # scaled to test size: 8 ranks x 6 tasks, every result against the oracle.
    w = synth.stress_mix(ranks=8, per_rank=6, vadd_median=4096, side_median=96)
    run_workload(gvm, w, mode=mode, path=path, depth=8, slice_mb=32)


def test_continuous_solo_equals_mix_bitwise(gvm):
    """Serving (continuous mode): tasks of four ranks arrive open loop, 50 us
    apart per rank, while earlier ones are still on the GPU (the resident
    scheduler admits them as ring slots and staging space free up). Every
    result must be bitwise the one the same task gives when it runs alone
    through a manager of the same configuration, and the oracle's."""
    R, per = 4, 8
    w = synth.stress_mix(ranks=R, per_rank=per, vadd_median=1 << 18, side_median=320, rate_per_rank_hz=20000.0)
    cfg = dict(ring_depth=4, mode="continuous", sgemm_path="split3", slice_bytes=320 << 20)

    def task_of(spec, keep):
        t = gvm.GvmTask()
        if spec.kind == synth.TASK_VADD:
            a, b = synth.vadd_inputs(spec.seed, spec.n)
            ins = (pinned(a), pinned(b))
            out = torch.full((spec.n,), float("nan")).pin_memory()
            t.type, t.n = gvm.GVM_TASK_VADD, spec.n
        else:
            A, B = synth.sgemm_inputs(spec.seed, spec.m, spec.n, spec.k)
            ins = (pinned(A), pinned(B))
            out = torch.full((spec.m, spec.n), float("nan")).pin_memory()
            t.type, t.m, t.n, t.k = gvm.GVM_TASK_SGEMM, spec.m, spec.n, spec.k
        t.flags = 0
        t.a, t.b, t.c = ins[0].data_ptr(), ins[1].data_ptr(), out.data_ptr()
        keep.append(ins)
        return t, out

    keep, mix_out = [], {}
    with gvm.Manager(R, **cfg) as mgr:
        ranks = [mgr.attach(r) for r in range(R)]
        by_rank = w.by_rank()
        arrays, arrivals = [], []
        for r in range(R):
            arr = (gvm.GvmTask * per)()
            for i, spec in enumerate(by_rank[r]):
                arr[i], mix_out[(r, i)] = task_of(spec, keep)
            arrays.append(arr)
            arrivals.append([int(s.arrival_s * 1e9) for s in by_rank[r]])
        span, lat = mgr.open_loop_run(ranks, arrays, arrivals, max_inflight=4)
        assert mgr.stats()["device_status"] == 0
        # The mix overlapped: some task completed after a later arrival of another rank.
        done_at = [arrivals[r][i] / 1e9 + lat[r][i] for r in range(R) for i in range(per)]
        assert max(done_at) > min(a for arr in arrivals for a in arr[1:]) / 1e9
    with gvm.Manager(1, **cfg) as solo:
        rk = solo.attach(0)
        for r in range(R):
            for i, spec in enumerate(w.by_rank()[r]):
                t, out = task_of(spec, keep)
                rk.sync(rk.submit(t))
                got = mix_out[(r, i)].numpy()
                assert np.array_equal(bits(got), bits(out.numpy())), spec
        assert solo.stats()["device_status"] == 0
    for spec in w.tasks:
        inputs = (synth.vadd_inputs(spec.seed, spec.n) if spec.kind == synth.TASK_VADD
                  else synth.sgemm_inputs(spec.seed, spec.m, spec.n, spec.k))
        check_result(spec, inputs, mix_out[(spec.rank, spec.index)])


@pytest.mark.parametrize("mode", ["barrier", "continuous"])
def test_tma_form_equals_fused_bitwise(gvm, mode):
    """The TMA form (binary32 A and B landed by tensor copies, split in place;
    tasks without maps staged by the converting warps' own loads) computes
    every element as the fused form does: equal bit for bit, on interior and
    ragged tiles, k below one k-step, n a multiple of 32 (B in one 3D box per
    k-step, slabs beyond n zero-filled: n = 384, 640), n a multiple of 4 only
    (eight 2D boxes), k and n not multiples of 4 (no maps), several tiles per
    CTA, and within the SGEMM rule against the oracle."""
    shapes = [(512, 512, 512), (128, 256, 32), (130, 260, 100), (300, 1000, 160), (257, 384, 200),
              (64, 700, 33), (1, 257, 31), (200, 192, 96), (1000, 520, 2052), (129, 257, 513), (256, 128, 4),
              (384, 640, 44), (640, 768, 1024)]
    w = synth.Workload("tma", 2)
    for i, (m, n, k) in enumerate(shapes):
        w.tasks.append(synth.TaskSpec(i % 2, i // 2, synth.TASK_SGEMM, m=m, n=n, k=k, seed=synth.task_seed(21, i)))
    fused = run_workload(gvm, w, mode=mode, path="split3", slice_mb=256)
    tma = run_workload(gvm, w, mode=mode, path="split3_tma", slice_mb=256)
    for spec in w.tasks:
        key = (spec.rank, spec.index)
        assert np.array_equal(bits(tma[key].numpy()), bits(fused[key].numpy())), spec
