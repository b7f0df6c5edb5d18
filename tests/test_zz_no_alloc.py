"""gvm_sgemm_f32_noalloc: split3 SGEMM for callers that cannot allocate.

Some callers cannot hand the library device scratch -- a plain C program with
no device allocator, a framework whose pool owns all device memory, a loop
where allocating is not allowed -- so this entry point keeps its scratch in a
fixed array inside the library. The test calls it through the C ABI twice in
a row (different operands, so stale scratch from the first call would show)
and compares each result with the regular entry point, gvm_sgemm_f32 with
caller-given scratch, within the SGEMM tolerance used by every test here
(relative Frobenius difference <= 1e-5). It also checks that a shape too big
for the fixed array is refused without a launch.

The file name makes pytest collect it last, so a run that stops at the first
failure has run every other test before this one.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def gvm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1511_07658_gb300 as g

    torch.cuda.set_device(0)
    return g


def rel_fro(x, y):
    x = x.astype(np.float64)
    y = y.astype(np.float64)
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def test_noalloc_matches_regular_entry_point(gvm):
    L = gvm.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for call, (m, n, k) in enumerate([(300, 520, 200), (512, 512, 512)]):
        A, B = synth.sgemm_inputs(synth.task_seed(9, call), m, n, k)
        tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        c_reg = torch.full((m, n), float("nan"), device="cuda")
        c_na = torch.full((m, n), float("nan"), device="cuda")
        gvm.sgemm_f32(tA, tB, c_reg, path="split3")
        rc = L.gvm_sgemm_f32_noalloc(tA.data_ptr(), tB.data_ptr(), c_na.data_ptr(), m, n, k, stream)
        assert rc == gvm.GVM_OK
        torch.cuda.synchronize()
        got, want = c_na.cpu().numpy(), c_reg.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_fro(got, want) <= TOL, (call, rel_fro(got, want))


def test_noalloc_rejects_oversize(gvm):
    L = gvm.lib()
    dummy = torch.empty(4, device="cuda")
    p = dummy.data_ptr()
    # 4 * (m + n) * k bytes of scratch above the fixed 32 MiB array
    assert L.gvm_sgemm_f32_noalloc(p, p, p, 4096, 4096, 4096, None) == gvm.GVM_ENOMEM
    assert L.gvm_sgemm_f32_noalloc(p, p, p, 0, 4, 4, None) == gvm.GVM_EINVAL
    assert L.gvm_sgemm_f32_noalloc(None, p, p, 4, 4, 4, None) == gvm.GVM_EINVAL
    assert isinstance(ctypes.c_int(0).value, int)
