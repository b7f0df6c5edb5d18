"""The SGEMM acceptance rule (``sgemm_bounds``) checked on the CPU against a
numpy emulation of the split arithmetic: it must accept every correct split
result, including single-product tasks whose error exceeds the 1e-5
statistical tolerance, and reject results with a missing product or term."""
import numpy as np
import pytest

import oracle
import synth
from sgemm_bounds import SampledCheck, check_sgemm, gamma, sample_indices


def rn_bf16(x):
    """Round binary32 to the nearest bf16 (ties to even), kept in binary32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def split3_emulated(A, B, products=("lh", "hl", "hh"), skip_k=None):
    """C[i, j] = sum over k of the kept bf16 products, each exact, added in
    binary32 in k order (the device's order of products within a k slice is
    lo*hi, hi*lo, hi*hi)."""
    Ah = rn_bf16(A)
    Al = rn_bf16(A - Ah)
    Bh = rn_bf16(B)
    Bl = rn_bf16(B - Bh)
    parts = {"lh": (Al, Bh), "hl": (Ah, Bl), "hh": (Ah, Bh), "ll": (Al, Bl)}
    m, k = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), np.float32)
    for kk in range(k):
        if kk == skip_k:
            continue
        for name in products:
            X, Y = parts[name]
            p = (X[:, kk : kk + 1].astype(np.float64) * Y[kk : kk + 1, :].astype(np.float64)).astype(np.float32)
            C = (C + p).astype(np.float32)
    return C


def test_split_residual_is_below_2_pow_16():
    a, _ = synth.vadd_inputs(3, 1 << 16)
    a = a[a != 0]
    h = rn_bf16(a)
    lo = rn_bf16(a - h)
    r = np.abs(a.astype(np.float64) - h - lo) / np.abs(a)
    assert r.max() <= 2.0 ** -16


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 2), (3, 2, 1), (5, 7, 3), (16, 16, 64), (17, 19, 512)])
def test_rule_accepts_split_results(shape):
    m, n, k = shape
    worst = 0.0
    for seed in range(200 if m * n < 4 else 10):
        A, B = synth.sgemm_inputs(9000 + seed, m, n, k)
        C = split3_emulated(A, B)
        check_sgemm(C, A, B)
        worst = max(worst, oracle.rel_fro_err(C, oracle.sgemm64(A, B)))
    if m * n * k == 1:
        # single products: the error does exceed the statistical 1e-5 for
        # some inputs, which is why that check needs many elements
        assert 1e-5 < worst < gamma(1)


@pytest.mark.parametrize(
    "mutant",
    [
        dict(products=("hh",)),
        dict(products=("lh", "hh")),
        dict(products=("hl", "hh")),
        dict(skip_k=0),
    ],
)
def test_rule_rejects_missing_terms(mutant):
    A, B = synth.sgemm_inputs(77, 6, 5, 9)
    with pytest.raises(AssertionError):
        check_sgemm(split3_emulated(A, B, **mutant), A, B)


def test_rule_rejects_transposed_and_sign_errors():
    A, B = synth.sgemm_inputs(78, 8, 8, 8)
    C = split3_emulated(A, B)
    with pytest.raises(AssertionError):
        check_sgemm(C.T.copy(), A, B)
    with pytest.raises(AssertionError):
        check_sgemm(-C, A, B)


def test_sampled_rule_accepts_split_results_and_keeps_edges():
    rng = np.random.default_rng(5)
    chk = SampledCheck()
    for seed, (m, n, k) in enumerate([(40, 36, 64), (130, 257, 65), (3, 300, 17)]):
        A, B = synth.sgemm_inputs(9100 + seed, m, n, k)
        C = split3_emulated(A, B)
        rows, cols = sample_indices(rng, m, 8), sample_indices(rng, n, 8)
        assert rows[0] == 0 and rows[-1] == m - 1 and cols[0] == 0 and cols[-1] == n - 1
        assert len(set(rows)) == len(rows) == min(m, 8)
        chk.add(C, A, B, rows, cols)
    assert chk.finish() < 1e-5


def test_sampled_rule_rejects_a_wrong_sample_and_a_transpose():
    rng = np.random.default_rng(6)
    A, B = synth.sgemm_inputs(9200, 24, 24, 32)
    C = split3_emulated(A, B)
    rows, cols = sample_indices(rng, 24, 6), sample_indices(rng, 24, 6)
    bad = C.copy()
    bad[rows[2], cols[3]] *= 1.001
    with pytest.raises(AssertionError):
        SampledCheck().add(bad, A, B, rows, cols)
    with pytest.raises(AssertionError):
        SampledCheck().add(C.T.copy(), A, B, rows, cols)
    with pytest.raises(AssertionError):
        SampledCheck().add(split3_emulated(A, B, products=("hh",)), A, B, rows, cols)
