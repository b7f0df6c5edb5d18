"""One client process of the cross-process GPU tests (no CUDA here): opens
its rank of a served region, writes seeded inputs into its data area, submits,
arrives at the request barrier, waits and checks every result against the CPU
oracle. Exit status 0 = every check passed.

    python tests/ipc_worker.py <name> <rank> <scenario>

Scenarios: mix (vector add, vector multiply, ragged and 512^3 SGEMM, two
barrier steps), late (mix, opened 3 s after the others started: it joins a
later request barrier), bad (a task whose result would leave the data area: refused,
the task before it completes), vanish (submits, then ends without the
barrier or closing).
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from paper_1511_07658_gb300 import GVM_EINVAL  # noqa: E402
from paper_1511_07658_gb300.ipc import IpcClient  # noqa: E402
from sgemm_bounds import check_sgemm  # noqa: E402


def al(x):
    return (x + 255) // 256 * 256


def bits(x):
    return np.ascontiguousarray(x).view(np.uint32)


def mix(c, rank, steps=2):
    specs = [("vadd", 70001 + rank), ("vmul", 4099 + rank), ("sgemm", (130, 257, 65)), ("sgemm", (512, 512, 512))]
    for step in range(steps):
        off = 0
        jobs = []
        for i, (kind, shape) in enumerate(specs):
            seed = synth.task_seed(rank, 100 * step + i)
            if kind == "sgemm":
                m, n, k = shape
                A, B = synth.sgemm_inputs(seed, m, n, k)
                oa, ob, oc = off, off + al(A.nbytes), off + al(A.nbytes) + al(B.nbytes)
                off = oc + al(4 * m * n)
                c.floats(oa, A.size)[:] = A.ravel()
                c.floats(ob, B.size)[:] = B.ravel()
                seq = c.submit_sgemm(oa, ob, oc, m, n, k)
                jobs.append((seq, kind, (A, B), oc, m * n))
            else:
                n = shape
                a, b = synth.vmul_inputs(seed, n) if kind == "vmul" else synth.vadd_inputs(seed, n)
                oa, ob, oc = off, off + al(4 * n), off + 2 * al(4 * n)
                off = oc + al(4 * n)
                c.floats(oa, n)[:] = a
                c.floats(ob, n)[:] = b
                seq = c.submit_vmul(oa, ob, oc, n, 15) if kind == "vmul" else c.submit_vadd(oa, ob, oc, n)
                jobs.append((seq, kind, (a, b), oc, n))
        c.barrier()
        for seq, kind, inp, oc, cnt in jobs:
            c.wait(seq, timeout_s=60)
            out = c.floats(oc, cnt).copy()
            if kind == "vadd":
                assert np.array_equal(bits(out), bits(oracle.vadd(*inp))), (rank, step, kind)
            elif kind == "vmul":
                assert np.array_equal(bits(out), bits(oracle.vmul(inp[0], inp[1], 15))), (rank, step, kind)
            else:
                check_sgemm(out, inp[0], inp[1])


def bad(c, rank):
    n = 1000
    a, b = synth.vadd_inputs(7, n)
    c.floats(0, n)[:] = a
    c.floats(4096, n)[:] = b
    s0 = c.submit_vadd(0, 4096, 8192, n)
    s1 = c.submit_vadd(0, 4096, c.data_bytes - 8, n)  # result would leave the data area
    c.barrier()
    c.wait(s0, timeout_s=60)
    assert np.array_equal(bits(c.floats(8192, n)), bits(oracle.vadd(a, b)))
    assert c.wait_code(s1, timeout_s=60) == GVM_EINVAL


def main():
    name, rank, scenario = sys.argv[1], int(sys.argv[2]), sys.argv[3]
    if scenario == "late":
        time.sleep(3.0)
        scenario = "mix"
    c = IpcClient(name, rank)
    if scenario == "vanish":
        c.submit_vadd(0, 0, 0, 16)
        os._exit(0)
    {"mix": mix, "bad": bad}[scenario](c, rank)
    c.close()
    print("ok", rank, scenario)


if __name__ == "__main__":
    main()
