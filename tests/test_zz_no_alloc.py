"""gvm_sgemm_f32_noalloc: split3 SGEMM for callers that cannot allocate.

Some callers cannot hand the library device scratch -- a plain C program with
no device allocator, a framework whose pool owns all device memory, a loop
where allocating is not allowed -- so this entry point keeps its scratch in a
fixed array inside the library.

The test calls it through the C ABI twice in a row on the one shared array:
first a large shape, then a smaller one whose k is not a multiple of 8, so
that the second call runs on scratch still holding the first call's planes
(padding columns included). Both calls run the same split pass and the same
tensor-core kernel as the regular entry point (gvm_sgemm_f32 on the split3
path with caller-given scratch), so each result must equal that entry
point's bit for bit, and each must be within the SGEMM acceptance rule
against the binary64 oracle. It also checks that refused calls launch
nothing.

The file name makes pytest collect it last, so a run that stops at the first
failure has run every other test before this one.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from sgemm_bounds import check_sgemm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gvm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1511_07658_gb300 as g

    torch.cuda.set_device(0)
    return g


def test_noalloc_matches_regular_entry_point(gvm):
    L = gvm.lib()
    stream = torch.cuda.current_stream().cuda_stream
    # large first, then a smaller shape with k % 8 != 0 on the stale array
    for call, (m, n, k) in enumerate([(512, 512, 512), (300, 520, 203)]):
        A, B = synth.sgemm_inputs(synth.task_seed(9, call), m, n, k)
        tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        c_reg = torch.full((m, n), float("nan"), device="cuda")
        c_na = torch.full((m, n), float("nan"), device="cuda")
        gvm.sgemm_f32(tA, tB, c_reg, path="split3")
        rc = L.gvm_sgemm_f32_noalloc(tA.data_ptr(), tB.data_ptr(), c_na.data_ptr(), m, n, k, stream)
        assert rc == gvm.GVM_OK
        torch.cuda.synchronize()
        got, want = c_na.cpu().numpy(), c_reg.cpu().numpy()
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), call
        check_sgemm(got, A, B, oracle.sgemm64(A, B))


def test_noalloc_refusals_launch_nothing(gvm):
    L = gvm.lib()
    c = torch.full((4, 4), 7.0, device="cuda")
    p = c.data_ptr()
    # 4 * (m + n) * kp bytes of scratch above the fixed 32 MiB array
    assert L.gvm_sgemm_f32_noalloc(p, p, p, 4096, 4096, 4096, None) == gvm.GVM_ENOMEM
    assert L.gvm_sgemm_f32_noalloc(p, p, p, 0, 4, 4, None) == gvm.GVM_EINVAL
    assert L.gvm_sgemm_f32_noalloc(None, p, p, 4, 4, 4, None) == gvm.GVM_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(c, torch.full((4, 4), 7.0, device="cuda"))
