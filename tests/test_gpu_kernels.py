"""Parity of the task kernels alone (gvm_vadd_f32, gvm_vmul_f32,
gvm_sgemm_f32) against the CPU oracle, through the C ABI. Vector add and
vector multiply: bit-exact. SGEMM: within the elementwise bound of the split
arithmetic and, for results of 256 elements or more, relative Frobenius
error <= 1e-5 against the binary64 oracle (``sgemm_bounds``); exact on
integer operands whose products and sums are exact in both arithmetics."""
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


@pytest.mark.parametrize("n", [0, 1, 3, 4097, 65536, 65536 + 3, (1 << 22) + 5])
def test_vadd_bitexact(gvm, n):
    a, b = synth.vadd_inputs(synth.task_seed(7, n % 1000), n)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    tc = torch.full_like(ta, float("nan"))
    gvm.vadd_f32(ta, tb, tc)
    torch.cuda.synchronize()
    assert np.array_equal(bits(tc.cpu().numpy()), bits(oracle.vadd(a, b)))


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_vadd_misaligned(gvm, shift):
    n = 100003
    a, b = synth.vadd_inputs(99, n + 8)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    tc = torch.zeros(n + 8, device="cuda")
    gvm.vadd_f32(ta[shift : shift + n], tb[(shift + 1) % 4 : (shift + 1) % 4 + n], tc[shift : shift + n])
    torch.cuda.synchronize()
    want = oracle.vadd(a[shift : shift + n], b[(shift + 1) % 4 : (shift + 1) % 4 + n])
    got = tc.cpu().numpy()
    assert np.array_equal(bits(got[shift : shift + n]), bits(want))
    assert np.all(got[:shift] == 0) and np.all(got[shift + n :] == 0)


def test_vadd_ieee_cases(gvm, golden):
    rows = golden("vadd_ieee_cases.txt")
    a = np.array([int(r[0], 16) for r in rows], dtype=np.uint32).view(np.float32)
    b = np.array([int(r[1], 16) for r in rows], dtype=np.uint32).view(np.float32)
    want = np.array([int(r[2], 16) for r in rows], dtype=np.uint32)
    tc = torch.empty(len(rows), device="cuda")
    gvm.vadd_f32(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), tc)
    torch.cuda.synchronize()
    assert np.array_equal(bits(tc.cpu().numpy()), want)


@pytest.mark.parametrize("n,iters", [(0, 15), (1, 1), (4097, 15), (65536 + 3, 2), ((1 << 22) + 5, 15), (70001, 1024)])
def test_vmul_bitexact(gvm, n, iters):
    a, b = synth.vmul_inputs(synth.task_seed(9, n % 1000), n)
    if iters > 40:  # keep long products normal: b = 1 +- 2**-10
        b = (np.float32(1.0) + (b - np.float32(1.0)) * np.float32(2.0 ** -8)).astype(np.float32)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    tc = torch.full_like(ta, float("nan"))
    gvm.vmul_f32(ta, tb, tc, iters)
    torch.cuda.synchronize()
    assert np.array_equal(bits(tc.cpu().numpy()), bits(oracle.vmul(a, b, iters)))


@pytest.mark.parametrize("shift", [1, 3])
def test_vmul_misaligned(gvm, shift):
    n = 100003
    a, b = synth.vmul_inputs(98, n + 8)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    tc = torch.zeros(n + 8, device="cuda")
    gvm.vmul_f32(ta[shift : shift + n], tb[(shift + 1) % 4 : (shift + 1) % 4 + n], tc[shift : shift + n], 15)
    torch.cuda.synchronize()
    want = oracle.vmul(a[shift : shift + n], b[(shift + 1) % 4 : (shift + 1) % 4 + n], 15)
    got = tc.cpu().numpy()
    assert np.array_equal(bits(got[shift : shift + n]), bits(want))
    assert np.all(got[:shift] == 0) and np.all(got[shift + n :] == 0)


def test_vmul_rejects_bad_iters(gvm):
    t = torch.zeros(16, device="cuda")
    for iters in (0, 1025):
        with pytest.raises(RuntimeError):
            gvm.vmul_f32(t, t, t, iters)


SHAPES = [
    (1, 1, 1),
    (5, 7, 3),
    (64, 64, 64),
    (128, 256, 32),
    (200, 136, 96),
    (257, 130, 67),
    (300, 520, 1000),
    (512, 512, 512),
    (129, 257, 513),
]


def run_sgemm(gvm, A, B, path):
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    tC = torch.full((A.shape[0], B.shape[1]), float("nan"), device="cuda")
    gvm.sgemm_f32(tA, tB, tC, path=path)
    torch.cuda.synchronize()
    return tC.cpu().numpy()


@pytest.mark.parametrize("path", ["fma", "split3", "split3_fused", "split3_wide"])
@pytest.mark.parametrize("shape", SHAPES)
def test_sgemm_normal_inputs(gvm, path, shape):
    m, n, k = shape
    A, B = synth.sgemm_inputs(synth.task_seed(m, n % 1000), m, n, k)
    C = run_sgemm(gvm, A, B, path)
    check_sgemm(C, A, B)
    from paper_1511_07658_gb300.manager import kernel_status

    assert kernel_status() == 0


@pytest.mark.parametrize("path", ["fma", "split3", "split3_fused", "split3_wide"])
@pytest.mark.parametrize("shape", [(9, 11, 64), (130, 260, 100), (256, 256, 256)])
def test_sgemm_integer_exact(gvm, path, shape):
    # |x| <= 16 and K <= 256: every product and partial sum is an integer
    # below 2^24, exact in binary32, and bf16 holds the operands exactly.
    m, n, k = shape
    A, B = synth.sgemm_int_inputs(1234 + k, m, n, k)
    C = run_sgemm(gvm, A, B, path)
    exact = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    assert np.array_equal(C.astype(np.float64), exact)


def test_split3_identity_closed_form(gvm):
    # B = I: split3 returns Ah + Al (the dropped lo*lo term multiplies by 0),
    # which differs from A by at most 2^-16 relative per element (two
    # roundings to 8-bit significands, unit roundoff 2^-8 each).
    m = k = 192
    A, _ = synth.sgemm_inputs(77, m, k, k)
    C = run_sgemm(gvm, A, np.eye(k, dtype=np.float32), "split3")
    rel = np.abs(C.astype(np.float64) - A) / np.maximum(np.abs(A.astype(np.float64)), 1e-30)
    assert rel.max() <= 2.0 ** -16
    assert np.any(C != A)  # the residual below the two bf16 pieces is dropped


def test_fma_identity_exact(gvm):
    A, _ = synth.sgemm_inputs(78, 100, 60, 60)
    C = run_sgemm(gvm, A, np.eye(60, dtype=np.float32), "fma")
    assert np.array_equal(C, A)


@pytest.mark.parametrize(
    "shape",
    [(128, 256, 32), (257, 130, 67), (512, 512, 512), (129, 257, 513), (300, 1001, 77),
     (130, 260, 100), (1000, 520, 2052), (4096, 2048, 96), (2500, 3000, 40)],
)
def test_split3_fused_equals_prepass(gvm, shape):
    # Same split rule, same products in the same order per 16-wide k slice,
    # same tile shape: the fused staging must give the pre-pass result bit for
    # bit. The large shapes give several tiles per CTA (both accumulators and
    # the stage ring wrap), the odd ones ragged tiles and rows aligned to 4,
    # 8 or 16 bytes only (each load width of the converters).
    m, n, k = shape
    A, B = synth.sgemm_inputs(synth.task_seed(7, m % 1000), m, n, k)
    C1 = run_sgemm(gvm, A, B, "split3")
    C2 = run_sgemm(gvm, A, B, "split3_fused")
    assert np.array_equal(bits(C1), bits(C2)), shape
    from paper_1511_07658_gb300.manager import kernel_status

    assert kernel_status() == 0


@pytest.mark.parametrize(
    "shape",
    [(256, 256, 32), (257, 130, 67), (512, 512, 512), (129, 257, 513), (300, 1001, 77),
     (130, 260, 100), (1000, 520, 2052), (4096, 2048, 96), (2500, 3000, 40), (256, 256, 1),
     (768, 1024, 512), (1024, 512, 2048), (512, 768, 64), (520, 512, 256), (200, 300, 96), (384, 640, 44)],
)
def test_split3_wide_equals_prepass(gvm, shape):
    # 256 x 256 tiles of one CTA (two 128-row MMA halves sharing each B stage,
    # one accumulator drained after the next tile's first k-step): the same
    # products in the same order per element, so the pre-pass result bit for
    # bit. k = 1 and k = 32 leave one group without a k-step of a tile.
    # Where k is a multiple of 4, A arrives by TMA boxes into the landing
    # buffers, rows and k beyond A zero-filled (m = 200: a box taller than A;
    # k = 44: a partial last k-step); several tiles per CTA check that the
    # landings of consecutive tiles alternate correctly.
    m, n, k = shape
    A, B = synth.sgemm_inputs(synth.task_seed(11, m % 1000), m, n, k)
    C1 = run_sgemm(gvm, A, B, "split3")
    C2 = run_sgemm(gvm, A, B, "split3_wide")
    assert np.array_equal(bits(C1), bits(C2)), shape
    from paper_1511_07658_gb300.manager import kernel_status

    assert kernel_status() == 0


