"""Cross-process rank segments without a GPU: creation, naming, the request
ring, the barrier counters, attachment rules and liveness, exercised from
child processes (no manager is serving, so nothing runs)."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def g():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1511_07658_gb300 as g

    return g


def uniq(tag):
    return f"gvmt-{tag}-{os.getpid()}"


def run_child(code, *args):
    """Runs `code` in a fresh Python process (the package importable)."""
    src = "import sys\nsys.path.insert(0, %r)\n" % ROOT + textwrap.dedent(code)
    return subprocess.run([sys.executable, "-c", src, *map(str, args)], capture_output=True, text=True, timeout=120)


def test_create_rejects_bad_arguments(g):
    from paper_1511_07658_gb300.ipc import IpcRegion

    for name, nranks, nbytes, depth in [("bad/name", 1, 1 << 20, 8), ("", 1, 1 << 20, 8), ("ok", 0, 1 << 20, 8),
                                         ("ok", 1, 0, 8), ("ok", 1, 1 << 20, 6), ("x" * 41, 1, 1 << 20, 8)]:
        with pytest.raises(RuntimeError):
            IpcRegion.create(name, nranks, nbytes, depth)


def test_create_twice_and_open_missing(g):
    from paper_1511_07658_gb300 import GVM_EBUSY, GVM_EINVAL
    from paper_1511_07658_gb300._abi import GvmError
    from paper_1511_07658_gb300.ipc import IpcClient, IpcRegion

    name = uniq("dup")
    reg = IpcRegion.create(name, 2, 1 << 20, 8)
    try:
        with pytest.raises(GvmError) as e:
            IpcRegion.create(name, 2, 1 << 20, 8)
        assert e.value.code == GVM_EBUSY
        with pytest.raises(GvmError) as e:
            IpcClient(name, 2)  # no such rank
        assert e.value.code == GVM_EINVAL
    finally:
        reg.destroy()
    with pytest.raises(GvmError) as e:
        IpcClient(name, 0)  # unlinked
    assert e.value.code == GVM_EINVAL


def test_child_requests_barrier_and_data_are_shared(g):
    from paper_1511_07658_gb300 import GVM_IPC_CLOSED, GVM_TASK_SGEMM, GVM_TASK_VADD
    from paper_1511_07658_gb300.ipc import IpcClient, IpcRegion

    name = uniq("child")
    reg = IpcRegion.create(name, 3, 4 << 20, 8)
    try:
        r = run_child(
            """
            import numpy as np
            from paper_1511_07658_gb300.ipc import IpcClient
            c = IpcClient(sys.argv[1], 1)
            x = c.floats(0, 1000)
            x[:] = np.arange(1000, dtype=np.float32)
            s0 = c.submit_vadd(0, 4000, 8000, 1000)
            s1 = c.submit_sgemm(0, 65536, 131072, 16, 16, 16)
            c.barrier()
            s2 = c.submit_vmul(0, 4000, 8000, 1000, 15)
            print(s0, s1, s2)
            c.close()
            """,
            name,
        )
        assert r.returncode == 0, r.stderr
        assert r.stdout.split() == ["0", "1", "2"]
        st = reg.peek(1)
        assert st == {"head": 3, "arrived": 1, "done": 0, "state": GVM_IPC_CLOSED}
        assert reg.peek(0)["state"] == 0 and reg.peek(2)["head"] == 0
        # A closed rank can be opened again; its data area kept the child's writes.
        c = IpcClient(name, 1)
        assert np.array_equal(c.floats(0, 1000), np.arange(1000, dtype=np.float32))
        assert c.data_bytes % (2 << 20) == 0
        c.close()
    finally:
        reg.destroy()


def test_ring_full_busy_and_timeout(g):
    from paper_1511_07658_gb300 import GVM_EAGAIN, GVM_EBUSY, GVM_ETIMEDOUT
    from paper_1511_07658_gb300._abi import GvmError
    from paper_1511_07658_gb300.ipc import IpcClient, IpcRegion

    name = uniq("full")
    reg = IpcRegion.create(name, 1, 1 << 20, 4)
    try:
        c = IpcClient(name, 0)
        with pytest.raises(GvmError) as e:
            IpcClient(name, 0)  # this (live) process holds it
        assert e.value.code == GVM_EBUSY
        seqs = [c.submit_vadd(0, 0, 0, 16) for _ in range(4)]
        assert seqs == [0, 1, 2, 3]
        with pytest.raises(GvmError) as e:
            c.submit_vadd(0, 0, 0, 16)  # nobody takes requests: the ring of 4 is full
        assert e.value.code == GVM_EAGAIN
        assert c.wait_code(0, timeout_s=0.05) == GVM_ETIMEDOUT
        c.close()
    finally:
        reg.destroy()


def test_rank_of_an_ended_process_can_be_taken(g):
    from paper_1511_07658_gb300 import GVM_IPC_ATTACHED
    from paper_1511_07658_gb300.ipc import IpcClient, IpcRegion

    name = uniq("lost")
    reg = IpcRegion.create(name, 1, 1 << 20, 8)
    try:
        r = run_child(
            """
            import os
            from paper_1511_07658_gb300.ipc import IpcClient
            c = IpcClient(sys.argv[1], 0)
            c.submit_vadd(0, 0, 0, 4)
            os._exit(0)  # ends without closing
            """,
            name,
        )
        assert r.returncode == 0, r.stderr
        assert reg.peek(0)["state"] == GVM_IPC_ATTACHED
        c = IpcClient(name, 0)  # the holder has ended
        assert reg.peek(0)["head"] == 1
        c.close()
    finally:
        reg.destroy()
