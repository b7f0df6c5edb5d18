"""Cross-process ranks on the GPU: client processes (tests/ipc_worker.py, no
CUDA) share one manager through their shared-memory segments; every result is
checked against the CPU oracle inside the client."""
import os
import subprocess
import sys

import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
WORKER = os.path.join(HERE, "ipc_worker.py")


@pytest.fixture(scope="module")
def gvm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1511_07658_gb300 as g

    torch.cuda.set_device(0)
    return g


def run_clients(gvm, mode, scenarios, path="split3"):
    name = f"gvmg-{mode}-{os.getpid()}-{len(scenarios)}"
    nranks = len(scenarios) + 1  # the last rank never opens: not part of the barrier
    region = gvm.IpcRegion.create(name, nranks, 16 << 20, 16)
    try:
        with gvm.Manager(nranks, ring_depth=16, mode=mode, sgemm_path=path, slice_bytes=48 << 20) as mgr:
            server = gvm.IpcServer(mgr, region)
            try:
                procs = [subprocess.Popen([sys.executable, WORKER, name, str(r), sc], stdout=subprocess.PIPE,
                                          stderr=subprocess.PIPE, text=True) for r, sc in enumerate(scenarios)]
                outs = [p.communicate(timeout=240) for p in procs]
                counts = server.counts()
            finally:
                server.stop()
        for p, (o, e), sc in zip(procs, outs, scenarios):
            assert p.returncode == 0, (sc, e[-3000:])
        return counts
    finally:
        region.destroy()


@pytest.mark.parametrize("mode", ["barrier", "continuous", "ps1"])
def test_client_processes_share_the_gpu(gvm, mode):
    counts = run_clients(gvm, mode, ["mix", "mix", "mix"])
    assert counts["taken"] == counts["completed"] == 3 * 4 * 2
    if mode != "continuous":
        assert counts["barriers"] >= 2


def test_a_client_that_joins_late(gvm):
    # The early clients run their first barrier without the late one, which
    # then joins the next barrier (its first arrival is its own, not one the
    # others' barrier already served).
    counts = run_clients(gvm, "barrier", ["mix", "mix", "late"])
    assert counts["taken"] == counts["completed"] == 3 * 4 * 2
    assert counts["barriers"] >= 3


def test_refused_task_and_a_client_that_vanishes(gvm):
    # rank 0 submits a task whose result would leave its data area (refused
    # with GVM_EINVAL; its earlier task runs); rank 1 ends without arriving
    # at the barrier or closing (the manager drops it from the barrier once
    # its process has ended); rank 2 runs its mix to completion.
    counts = run_clients(gvm, "barrier", ["bad", "vanish", "mix"])
    assert counts["completed"] >= 1 + 8


def test_shutdown_refused_while_served(gvm):
    # The serving thread drives the manager's ranks: gvm_shutdown refuses
    # (GVM_ESTATE, nothing freed) until gvm_ipc_stop, then succeeds.
    name = f"gvmg-guard-{os.getpid()}"
    region = gvm.IpcRegion.create(name, 2, 4 << 20, 4)
    try:
        mgr = gvm.Manager(2, ring_depth=4, mode="barrier", slice_bytes=16 << 20)
        server = gvm.IpcServer(mgr, region)
        with pytest.raises(gvm.GvmError) as e:
            mgr.shutdown()
        assert e.value.code == gvm.GVM_ESTATE
        assert mgr.handle is not None
        server.stop()
        mgr.shutdown()
        assert mgr.handle is None
    finally:
        region.destroy()
