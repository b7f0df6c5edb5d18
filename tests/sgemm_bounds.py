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


def sample_indices(rng, size: int, count: int) -> np.ndarray:
    """`count` distinct sorted indices of range(size), always holding the
    first and the last (the edges of the last, ragged tile)."""
    if size <= count:
        return np.arange(size)
    inner = rng.choice(np.arange(1, size - 1), count - 2, replace=False)
    return np.sort(np.concatenate([[0, size - 1], inner]))


class SampledCheck:
    """The acceptance rule on sampled outputs of many results, for sizes
    where the full binary64 product is too slow: each block C[rows][:, cols]
    is compared elementwise with the oracle's product A[rows] @ B[:, cols]
    (the same dot products the full product would form), and the relative
    Frobenius error is taken over all blocks together."""

    def __init__(self):
        self.C = []
        self.R = []
        self.worst = 0.0

    def add(self, C, A, B, rows, cols, label=""):
        self.add_block(np.asarray(C, dtype=np.float32)[np.ix_(rows, cols)], A, B, rows, cols, label)

    def add_block(self, Cs, A, B, rows, cols, label=""):
        """Cs = the result's entries at rows x cols, already gathered."""
        A = np.asarray(A, dtype=np.float32)
        B = np.asarray(B, dtype=np.float32)
        Ar = np.ascontiguousarray(A[rows])
        Bc = np.ascontiguousarray(B[:, cols])
        R = oracle.sgemm64(Ar, Bc)
        Cs = np.asarray(Cs, dtype=np.float32).reshape(len(rows), len(cols))
        k = A.shape[1]
        S = np.abs(Ar).astype(np.float64) @ np.abs(Bc).astype(np.float64)
        bound = gamma(k) * S + k * 2.0 ** -149
        worst = float(np.max(np.abs(Cs.astype(np.float64) - R) / bound)) if Cs.size else 0.0
        assert worst <= 1.0, f"{label}: elementwise split bound exceeded: worst |C - R| / bound = {worst:.3g}"
        self.worst = max(self.worst, worst)
        self.C.append(np.ascontiguousarray(Cs).reshape(-1))
        self.R.append(R.reshape(-1))

    def finish(self) -> float:
        """Relative Frobenius error over every sample (checked from 256)."""
        C = np.concatenate(self.C) if self.C else np.zeros(0, np.float32)
        R = np.concatenate(self.R) if self.R else np.zeros(0)
        if C.size == 0:
            return 0.0
        err = oracle.rel_fro_err(C, R)
        if C.size >= FRO_MIN_ELEMENTS:
            assert err <= FRO_TOL, f"relative Frobenius error over {C.size} samples {err:.3g} > {FRO_TOL}"
        return err
