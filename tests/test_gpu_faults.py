"""Failure detection without a GPU fault.

A bounded wait in the scheduler runs out on purpose: the input copies of a
task are held back on its rank's input stream (a bounded sleep kernel queued
ahead of them) for longer than the manager's wait limit, so the scheduler
finds the task published but never ready. It must record a timeout status in
host memory and stop; the host reports GVM_EDEVICE, reads the status, and
shuts the manager down with every stream released. Nothing faults, traps or
hangs: the sleep and the wait both end on their own.
"""
import pytest
import torch

pytestmark = pytest.mark.gpu

KWHERE_READY_WAIT = 1
KSTATUS_TIMEOUT = 1


@pytest.fixture(scope="module")
def gvm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1511_07658_gb300 as g

    torch.cuda.set_device(0)
    return g


def test_ready_wait_times_out(gvm):
    mgr = gvm.Manager(2, ring_depth=4, mode="barrier", sgemm_path="split3", slice_bytes=8 << 20,
                      wait_timeout_s=0.3)
    rk = mgr.attach(0)
    x = torch.ones(4096).pin_memory()
    out = torch.zeros(4096).pin_memory()
    # Hold rank 0's input stream for 3e9 SM cycles (about 1.5-2 s; bounded).
    cycles = int(3.0e9)
    with torch.cuda.stream(mgr.copy_streams[0]):
        torch.cuda._sleep(cycles)
    seq = rk.submit_vadd(x, x, out)
    mgr.flush()
    with pytest.raises(gvm.GvmError) as e:
        rk.sync(seq)
    assert e.value.code == gvm.GVM_EDEVICE
    st = mgr.stats()
    assert st["device_status"] == KSTATUS_TIMEOUT
    assert st["device_where"] == KWHERE_READY_WAIT
    with pytest.raises(gvm.GvmError) as e:
        mgr.shutdown()
    assert e.value.code == gvm.GVM_EDEVICE
    # The context is still usable afterwards.
    torch.cuda.synchronize()
    y = torch.ones(1000, device="cuda") * 3
    assert float(y.sum()) == 3000.0


def test_manager_usable_after_failed_one(gvm):
    """A fresh manager works after another one stopped on an error."""
    with gvm.Manager(1, ring_depth=4, slice_bytes=8 << 20) as mgr:
        rk = mgr.attach(0)
        x = torch.full((1000,), 1.5).pin_memory()
        out = torch.zeros(1000).pin_memory()
        seq = rk.submit_vadd(x, x, out)
        mgr.flush()
        rk.sync(seq)
        assert torch.all(out == 3.0)
