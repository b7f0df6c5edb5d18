"""Acceptance rule for a binary32 SGEMM result against the binary64 oracle.

Two checks, both derived from the arithmetic of the two device paths:

* Elementwise, always: |C - R| <= gamma(K) * (|A| |B|) + K * 2**-149, with
  gamma(K) = 3.1 * 2**-16 + 3 K * 2**-23.
  Split path: with hi = RN_bf16(x) and lo = RN_bf16(x - hi) (8-bit
  significands, unit roundoff 2**-8), |x - hi - lo| <= 2**-16 |x|. The
  three kept products hi*hi, hi*lo, lo*hi miss lo_a*lo_b and the two
  residual terms, each at most about 2**-16 |a b|: 3.1 * 2**-16 covers
  their sum with the (1 + 2**-8) factors. The 3 K exact bf16 products are
  summed in binary32; 3 K * 2**-23 bounds that sum's rounding even if each
  addition truncated. The FMA path (K fused multiply-adds in binary32) is
  well inside the same bound. The last term allows for subnormal flushes.
* Relative Frobenius error <= 1e-5 when the result has at least 256
  elements. This is a statistical tolerance: one element's split error can
  reach about 4.6e-5 of its magnitude, so with only a few outputs the norm
  is a small sample and only the elementwise bound applies.
"""
import numpy as np

import oracle

FRO_TOL = 1e-5
FRO_MIN_ELEMENTS = 256


def gamma(k: int) -> float:
    return 3.1 * 2.0 ** -16 + 3 * k * 2.0 ** -23


def check_sgemm(C, A, B, R=None):
    """Raises AssertionError (with the worst ratio) if C breaks either rule;
    returns the relative Frobenius error."""
    A = np.asarray(A, dtype=np.float32)
    B = np.asarray(B, dtype=np.float32)
    C = np.asarray(C, dtype=np.float32).reshape(A.shape[0], B.shape[1])
    if R is None:
        R = oracle.sgemm64(A, B)
    k = A.shape[1]
    S = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    bound = gamma(k) * S + k * 2.0 ** -149
    diff = np.abs(C.astype(np.float64) - R)
    worst = float(np.max(diff / bound)) if diff.size else 0.0
    assert worst <= 1.0, f"elementwise split bound exceeded: worst |C - R| / bound = {worst:.3g}"
    err = oracle.rel_fro_err(C, R)
    if C.size >= FRO_MIN_ELEMENTS:
        assert err <= FRO_TOL, f"relative Frobenius error {err:.3g} > {FRO_TOL}"
    return err
