"""Pins of the CPU oracle against facts fixed outside it (CPU only).

Each check ties the oracle to something other than itself: hand-derived IEEE
cases, a library routine (numpy), exact integer and rational arithmetic,
closed forms. The mutation tests at the end show that plausible mistakes in
the oracle (a transposed operand, a dropped term, a wrong sign, float32
accumulation, flush to zero) fail at least one pin.
"""
import math
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import model


def f32_bits(x):
    return np.asarray(x, dtype=np.float32).view(np.uint32)


def from_hex(h):
    return np.frombuffer(struct.pack("<I", int(h, 16)), dtype=np.float32)[0]


# ---------------------------------------------------------------- generators


def test_splitmix64_published_vectors(golden):
    for seed, i, val in golden("splitmix64_vectors.txt"):
        assert synth.splitmix64_scalar(int(seed), int(i)) == int(val)
        assert int(synth.splitmix64(int(seed), 1, int(i))[0]) == int(val)


def test_uniform_grid_and_range():
    x = synth.uniform_pm1(7, 100000)
    assert x.dtype == np.float32
    assert x.min() >= -1.0 and x.max() <= 1.0 - 2.0 ** -23
    k = (x.astype(np.float64) + 1.0) * 2.0 ** 23
    assert np.all(k == np.round(k))  # multiples of 2^-23
    assert abs(float(x.mean())) < 0.02


def test_normal_moments():
    x = synth.standard_normal(11, 200000).astype(np.float64)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01


def test_chunked_generation_matches_single_chunk():
    n = synth._CHUNK + 12345
    a = synth.uniform_pm1(3, n)
    b = np.concatenate([synth.uniform_pm1(3, synth._CHUNK), synth.uniform_pm1(3, 12345, synth._CHUNK)])
    assert np.array_equal(f32_bits(a), f32_bits(b))


# ---------------------------------------------------------------- vector add


def test_vadd_ieee_hand_cases(golden):
    rows = golden("vadd_ieee_cases.txt")
    a = np.array([from_hex(r[0]) for r in rows], dtype=np.float32)
    b = np.array([from_hex(r[1]) for r in rows], dtype=np.float32)
    want = np.array([int(r[2], 16) for r in rows], dtype=np.uint32)
    assert np.array_equal(f32_bits(oracle.vadd(a, b)), want)


def test_vadd_matches_numpy_float32():
    a, b = synth.vadd_inputs(synth.task_seed(3, 5), 65536)
    with np.errstate(all="ignore"):
        ref = np.add(a, b, dtype=np.float32)
    assert np.array_equal(f32_bits(oracle.vadd(a, b)), f32_bits(ref))


def test_vadd_empty():
    assert oracle.vadd(np.zeros(0, np.float32), np.zeros(0, np.float32)).size == 0


# ---------------------------------------------------------------- vector multiply


def _vmul_by_float64_rounding(a, b, iters):
    """Each binary32 product is exact in binary64 (24 + 24 bits < 53), so one
    cast back to binary32 is the single round-to-nearest-even of IEEE-754."""
    z = a.astype(np.float32)
    for _ in range(iters):
        z = (z.astype(np.float64) * b.astype(np.float64)).astype(np.float32)
    return z


@pytest.mark.parametrize("iters", [1, 2, 15, 40])
def test_vmul_matches_exact_product_rounded_once_per_step(iters):
    a, b = synth.vmul_inputs(synth.task_seed(2, iters), 40000)
    assert np.array_equal(f32_bits(oracle.vmul(a, b, iters)), f32_bits(_vmul_by_float64_rounding(a, b, iters)))


def test_vmul_one_product_is_numpy_float32_multiply():
    a, b = synth.vmul_inputs(synth.task_seed(4, 1), 65536)
    assert np.array_equal(f32_bits(oracle.vmul(a, b, 1)), f32_bits(np.multiply(a, b, dtype=np.float32)))


def test_vmul_powers_of_two_closed_form():
    # b = 2**e: every product is exact, so c = a * 2**(e * iters) exactly.
    a, _ = synth.vmul_inputs(synth.task_seed(5, 0), 4096)
    for e, iters in [(1, 15), (-1, 15), (3, 7), (0, 1024)]:
        b = np.full_like(a, np.float32(2.0 ** e))
        want = (a.astype(np.float64) * 2.0 ** (e * iters)).astype(np.float32)
        assert np.array_equal(f32_bits(oracle.vmul(a, b, iters)), f32_bits(want))


def test_vmul_small_cases_by_exact_rationals():
    # Brute force: exact rational product, rounded to the nearest binary32
    # (ties to even) by search among the two neighbours.
    a, b = synth.vmul_inputs(synth.task_seed(6, 0), 64)
    iters = 5
    got = oracle.vmul(a, b, iters)
    for i in range(a.size):
        z = np.float32(a[i])
        for _ in range(iters):
            exact = Fraction(float(z)) * Fraction(float(b[i]))
            lo = np.float32(float(exact))
            cands = {lo, np.nextafter(lo, np.float32(np.inf)), np.nextafter(lo, np.float32(-np.inf))}
            best = min(cands, key=lambda c: (abs(Fraction(float(c)) - exact), int(f32_bits(c)) & 1))
            z = best
        assert f32_bits(got[i]) == f32_bits(z)


def test_vmul_order_is_pinned():
    # Mutant: a * (b ** iters) with the power taken first; the rounding differs,
    # so the pins above would catch a wrong product order.
    a, b = synth.vmul_inputs(synth.task_seed(7, 0), 65536)
    p = np.ones_like(b)
    for _ in range(15):
        p = np.multiply(p, b, dtype=np.float32)
    mutant = np.multiply(a, p, dtype=np.float32)
    assert not np.array_equal(f32_bits(mutant), f32_bits(_vmul_by_float64_rounding(a, b, 15)))


def test_vmul_empty_and_limits():
    z = np.zeros(0, np.float32)
    assert oracle.vmul(z, z, 15).size == 0
    with pytest.raises(ValueError):
        oracle.vmul(z, z, 0)
    a, b = synth.vmul_inputs(synth.task_seed(8, 0), 1 << 16)
    assert a.min() >= -1.0 and a.max() < 1.0 and b.min() >= 0.75 and b.max() < 1.25
    c = oracle.vmul(a, b, 40)
    nz = c[a != 0]
    assert np.all(np.abs(nz) >= np.float32(2.0 ** -126))  # no subnormal on the recipe


# ---------------------------------------------------------------- matrix multiply


def sgemm_pins(fn):
    """All SGEMM pins as one predicate list; each entry is (name, passed)."""
    out = []
    rng = np.random.default_rng(0)
    # 1. numpy float64 matmul (library), elementwise within the fp64 bound.
    for (m, n, k) in [(7, 5, 3), (33, 17, 65), (64, 48, 200)]:
        A, B = synth.sgemm_inputs(synth.task_seed(1, m), m, n, k)
        C = fn(A, B)
        R = A.astype(np.float64) @ B.astype(np.float64)
        bound = 2 * k * 2.0 ** -53 * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64))
        out.append((f"numpy {m}x{n}x{k}", C.shape == R.shape and bool(np.all(np.abs(C - R) <= bound))))
    # 2. integer operands: the exact integer product.
    for (m, n, k) in [(9, 11, 64), (16, 3, 1), (5, 31, 17)]:
        A, B = synth.sgemm_int_inputs(99 + k, m, n, k)
        exact = A.astype(np.int64) @ B.astype(np.int64)
        C = fn(A, B)
        out.append((f"integer {m}x{n}x{k}", C.shape == exact.shape and bool(np.array_equal(C, exact.astype(np.float64)))))
    # 3. K = 1: the outer product, exact in binary64.
    a = rng.standard_normal((6, 1)).astype(np.float32)
    b = rng.standard_normal((1, 4)).astype(np.float32)
    out.append(("outer", bool(np.array_equal(fn(a, b), a.astype(np.float64) * b.astype(np.float64)))))
    # 4. B = I gives A; I on the left gives B.
    A = rng.standard_normal((5, 8)).astype(np.float32)
    out.append(("right identity", bool(np.array_equal(fn(A, np.eye(8, dtype=np.float32)), A.astype(np.float64)))))
    out.append(("left identity", bool(np.array_equal(fn(np.eye(5, dtype=np.float32), A), A.astype(np.float64)))))
    # 5. zero operand.
    out.append(("zero", bool(np.all(fn(np.zeros((3, 4), np.float32), A[:4, :6]) == 0.0))))
    # 6. brute force on tiny shapes: exact rationals within the ordered-sum
    #    bound, and a Python in-order binary64 sum bit for bit.
    ok_exact, ok_order = True, True
    for m in (1, 2, 3, 5):
        for n in (1, 2, 3, 5):
            for k in (1, 2, 3, 5):
                A, B = synth.sgemm_inputs(synth.task_seed(m, 10 * n + k), m, n, k)
                C = fn(A, B)
                if C.shape != (m, n):
                    ok_exact = ok_order = False
                    continue
                for i in range(m):
                    for j in range(n):
                        terms = [Fraction(float(A[i, t])) * Fraction(float(B[t, j])) for t in range(k)]
                        exact = sum(terms, Fraction(0))
                        mag = sum(abs(t) for t in terms)
                        if abs(Fraction(float(C[i, j])) - exact) > (k * Fraction(1, 2 ** 52)) * mag:
                            ok_exact = False
                        s = 0.0
                        for t in range(k):
                            s += float(A[i, t]) * float(B[t, j])
                        if s != float(C[i, j]):
                            ok_order = False
    out.append(("brute force exact", ok_exact))
    out.append(("brute force order", ok_order))
    return out


def test_sgemm64_pins():
    failed = [name for name, ok in sgemm_pins(oracle.sgemm64) if not ok]
    assert not failed, failed


def test_sgemm64_rejects_bad_shapes():
    with pytest.raises(ValueError):
        oracle.sgemm64(np.zeros((2, 3), np.float32), np.zeros((4, 2), np.float32))


def test_rel_fro_err_closed_forms():
    A, B = synth.sgemm_int_inputs(5, 8, 8, 8)
    R = oracle.sgemm64(A, B)
    C = R.astype(np.float32)  # integers, exact in float32
    assert oracle.rel_fro_err(C, R) == 0.0
    assert oracle.rel_fro_err(np.zeros_like(C), R) == 1.0
    scaled = (R * (1.0 + 2.0 ** -10)).astype(np.float32)  # exact: |R| small integers
    assert abs(oracle.rel_fro_err(scaled, R) - 2.0 ** -10) < 1e-15
    assert oracle.rel_fro_err(np.zeros(4, np.float32), np.zeros(4)) == 0.0
    assert math.isinf(oracle.rel_fro_err(np.ones(4, np.float32), np.zeros(4)))


# ---------------------------------------------------------------- mutations


def _mut_transpose_b(A, B):
    return oracle.sgemm64(A, B.T.copy()) if A.shape[1] == B.shape[1] else oracle.sgemm64(A, B).T.copy()


def _mut_drop_last_k(A, B):
    if A.shape[1] == 1:
        return np.zeros((A.shape[0], B.shape[1]))
    return oracle.sgemm64(A[:, :-1], B[:-1, :])


def _mut_f32_accumulate(A, B):
    C = np.zeros((A.shape[0], B.shape[1]), dtype=np.float32)
    for t in range(A.shape[1]):
        C += np.outer(A[:, t], B[t, :]).astype(np.float32)
    return C.astype(np.float64)


def _mut_sign(A, B):
    C = oracle.sgemm64(A, B)
    C[0, 0] = -C[0, 0]
    return C


def _mut_reverse_order(A, B):
    return oracle.sgemm64(A[:, ::-1].copy(), B[::-1, :].copy())


@pytest.mark.parametrize(
    "mutant", [_mut_transpose_b, _mut_drop_last_k, _mut_f32_accumulate, _mut_sign, _mut_reverse_order]
)
def test_sgemm_pins_catch_mutants(mutant):
    assert any(not ok for _, ok in sgemm_pins(mutant))


def test_vadd_pins_catch_ftz_and_truncation(golden):
    rows = golden("vadd_ieee_cases.txt")
    a = np.array([from_hex(r[0]) for r in rows], dtype=np.float32)
    b = np.array([from_hex(r[1]) for r in rows], dtype=np.float32)
    want = np.array([int(r[2], 16) for r in rows], dtype=np.uint32)
    # flush-to-zero mutant
    def ftz(x):
        x = x.copy()
        x[np.abs(x) < np.float32(2.0 ** -126)] = 0.0
        return x
    with np.errstate(all="ignore"):
        c_ftz = ftz(ftz(a) + ftz(b))
        # round-toward-zero mutant: exact sum in float64, truncated to float32
        s = a.astype(np.float64) + b.astype(np.float64)
        c_rz = s.astype(np.float32)
        over = np.abs(c_rz.astype(np.float64)) > np.abs(s)
        c_rz[over] = np.nextafter(c_rz[over], np.float32(0))
    assert not np.array_equal(f32_bits(c_ftz), want)
    assert not np.array_equal(f32_bits(c_rz), want)


# ---------------------------------------------------------------- execution model


def _params(seed, count):
    z = synth.splitmix64(seed, 5 * count)
    u = (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return [tuple(0.1 + 10.0 * u[5 * i : 5 * i + 5]) for i in range(count)]


def test_model_eq7_is_eq5_and_eq6():
    for t_init, t_in, t_comp, t_out, t_ctx in _params(1, 200):
        for n in (1, 2, 8, 16):
            assert math.isclose(
                model.t_total_ioi_ps2(n, t_in, t_comp, t_out),
                model.t_total_ioi_ps2_piecewise(n, t_in, t_comp, t_out),
                rel_tol=1e-12,
            )


def test_model_single_process_cases():
    for t_init, t_in, t_comp, t_out, t_ctx in _params(2, 100):
        alone = t_in + t_comp + t_out
        for f in (model.t_total_ci_ps1, model.t_total_ci_ps2, model.t_total_ioi_ps1, model.t_total_ioi_ps2):
            assert math.isclose(f(1, t_in, t_comp, t_out), alone, rel_tol=1e-12)
        assert math.isclose(model.t_total_no_vt(1, t_init, t_in, t_comp, t_out, t_ctx), t_init + alone, rel_tol=1e-12)


def test_model_speedup_limits():
    for p in _params(3, 50):
        big = 1e9
        assert math.isclose(model.speedup_ci(big, *p), model.speedup_max_ci(*p), rel_tol=1e-6)
        assert math.isclose(model.speedup_ioi(big, *p), model.speedup_max_ioi(*p), rel_tol=1e-6)


def test_model_policy_inequalities():
    # Style 2 never loses to style 1 for I/O-intensive tasks (Eq. 7 <= Eq. 4).
    for t_init, t_in, t_comp, t_out, t_ctx in _params(4, 200):
        for n in (1, 2, 8):
            assert model.t_total_ioi_ps2(n, t_in, t_comp, t_out) <= model.t_total_ioi_ps1(n, t_in, t_comp, t_out) + 1e-12
    # Style 1 beats style 2 for compute-bound tasks when the copies of one task
    # are shorter than its kernel (Eq. 2 < Eq. 3 iff T_in + T_out < T_comp).
    assert model.t_total_ci_ps1(8, 1.0, 5.0, 1.0) < model.t_total_ci_ps2(8, 1.0, 5.0, 1.0)
    assert model.t_total_ci_ps1(8, 2.0, 3.0, 2.0) > model.t_total_ci_ps2(8, 2.0, 3.0, 2.0)


def test_model_classes():
    assert model.classify(1, 5, 1) == model.CI
    assert model.classify(5, 1, 6) == model.IOI
    assert model.classify(5, 3, 1) == model.INTERMEDIATE
    assert model.classify(3, 3, 3) == model.CI  # boundary: <= is compute-intensive


def test_model_sequential_exceeds_shared():
    for t_init, t_in, t_comp, t_out, t_ctx in _params(5, 100):
        for n in (2, 4, 16):
            seq = model.t_total_no_vt(n, t_init, t_in, t_comp, t_out, t_ctx)
            assert seq > model.shared_time(n, t_in, t_comp, t_out)


def _pipeline_makespan(n, t_in, t_comp, t_out, servers):
    """Brute force: n identical tasks through input link -> kernel -> output
    link. Each link carries one copy at a time in task order; a kernel starts
    once its input has landed and one of ``servers`` kernel slots is free
    (slots taken in task order). Returns the time the last output lands."""
    free_in = 0.0
    slots = [0.0] * servers
    free_out = 0.0
    for j in range(n):
        landed = free_in + t_in
        free_in = landed
        s = min(range(servers), key=lambda i: slots[i])
        done = max(landed, slots[s]) + t_comp
        slots[s] = done
        free_out = max(free_out, done) + t_out
    return free_out


def test_model_duplex_closed_cases():
    # One task, one wave: its own chain, nothing overlaps.
    for t_init, t_in, t_comp, t_out, t_ctx in _params(6, 100):
        assert math.isclose(model.shared_time_duplex(1, t_in, t_comp, t_out, 1), t_in + t_comp + t_out, rel_tol=1e-12)
    # Compute-bound limit: no copies, every wave in turn.
    assert model.shared_time_duplex(16, 0.0, 3.0, 0.0, 5) == 15.0
    # Link-bound limit: no compute, the longer direction streams, one copy of
    # the shorter one is exposed.
    assert model.shared_time_duplex(8, 1.0, 0.0, 2.5, 1) == 8 * 2.5 + 1.0
    # Hand cases (worked by drawing the pipeline).
    assert model.shared_time_duplex(4, 1.0, 3.0, 2.0, 2) == 12.0
    assert model.shared_time_duplex(6, 1.0, 5.0, 1.0, 3) == 17.0
    assert model.shared_time_duplex(0, 1.0, 5.0, 1.0, 0) == 0.0


def test_model_duplex_against_pipeline_brute_force():
    # With one wave the variant is the makespan of the simulated pipeline and
    # equals Eq. 7; with several waves it is a lower bound on it.
    for t_init, t_in, t_comp, t_out, t_ctx in _params(7, 120):
        for n in (1, 2, 3, 8, 16):
            sim = _pipeline_makespan(n, t_in, t_comp, t_out, servers=n)
            duplex = model.shared_time_duplex(n, t_in, t_comp, t_out, 1)
            assert math.isclose(duplex, sim, rel_tol=1e-12)
            assert math.isclose(duplex, model.t_total_ioi_ps2(n, t_in, t_comp, t_out), rel_tol=1e-12)
            assert duplex <= model.t_total_ioi_ps1(n, t_in, t_comp, t_out) + 1e-12
            for servers in (1, 2, 5):
                w = model.waves(n, 1, servers, 1)
                sim = _pipeline_makespan(n, t_in, t_comp, t_out, servers)
                bound = model.shared_time_duplex(n, t_in, t_comp, t_out, w)
                assert bound <= sim + 1e-9
                # every resource's total busy time fits under it
                assert bound >= max(n * t_in, n * t_out, w * t_comp) - 1e-12
    # One slot serialises the kernels; with kernels longer than both copies
    # the compute chain is then the whole makespan.
    assert math.isclose(model.shared_time_duplex(5, 1.0, 4.0, 1.0, 5), _pipeline_makespan(5, 1.0, 4.0, 1.0, 1))


def test_model_duplex_pins_catch_mutants():
    def additive(n, t_in, t_c, t_out, w):
        return n * max(t_in, t_out) + w * t_c + min(t_in, t_out)

    def max_inside(n, t_in, t_c, t_out, w):
        return max(n * max(t_in, t_out), w * t_c) + min(t_in, t_out)

    for mut in (additive, max_inside):
        assert (mut(1, 1.0, 2.0, 3.0, 1) != 6.0 or mut(4, 1.0, 3.0, 2.0, 2) != 12.0
                or mut(6, 1.0, 5.0, 1.0, 3) != 17.0)


def test_model_waves_exact_ceiling():
    assert model.waves(0, 8, 152, 1) == 0
    assert model.waves(1, 1, 152, 1) == 1
    assert model.waves(19, 8, 152, 1) == 1  # 152 blocks: exactly one wave
    assert model.waves(20, 8, 152, 1) == 2  # 160 blocks: one over
    assert model.waves(152, 1, 152, 1) == 1
    assert model.waves(153, 1, 152, 1) == 2
    assert model.waves(304, 1, 152, 2) == 1
    assert model.waves(305, 1, 152, 2) == 2
    assert model.waves(1024, 8, 152, 1) == 54  # 8192 tiles of the 16 x 64 SGEMM 512^3 step
    with pytest.raises(ValueError):
        model.waves(1, 1, 0, 1)
    # brute force: the smallest w with w * slots >= blocks
    for blocks in range(0, 40):
        for slots in range(1, 9):
            w = 0
            while w * slots < blocks:
                w += 1
            assert model.waves(blocks, 1, slots, 1) == w


# ---------------------------------------------------------------- workloads


def test_rank_runner_is_order_and_isolation():
    w = synth.vadd_tiny(ranks=2, per_rank=3, n=1000)
    res = oracle.run_workload(w)
    for spec in w.tasks:
        a, b = synth.vadd_inputs(spec.seed, spec.n)
        assert np.array_equal(f32_bits(res[(spec.rank, spec.index)]), f32_bits(oracle.vadd(a, b)))


def test_workload_recipes():
    w = synth.serving_mix(ranks=16, total=4096)
    assert len(w.tasks) == 4096
    kinds = [t.kind for t in w.tasks]
    assert kinds.count(synth.TASK_VADD) == 2048
    for t in w.tasks:
        if t.kind == synth.TASK_VADD:
            assert 2 ** 16 <= t.n < 2 ** 24
        else:
            assert t.m == t.n == t.k and t.m in (256, 512, 1024, 2048)
    g = synth.grouped_mixed(ranks=4, per_rank=8)
    assert all(128 <= x <= 2048 and x % 64 == 0 for t in g.tasks for x in (t.m, t.n, t.k))


def test_stress_mix_recipe():
    # The stress recipe's own invariants: 70/30 mix within sampling noise,
    # clamps respected, arrivals increasing per rank, and the same draw every
    # time (seeded).
    w = synth.stress_mix(ranks=64, per_rank=32)
    kinds = [t.kind for t in w.tasks]
    frac = kinds.count(synth.TASK_VADD) / len(kinds)
    assert 0.65 < frac < 0.75
    for t in w.tasks:
        if t.kind == synth.TASK_VADD:
            assert 2 ** 10 <= t.n <= 2 ** 28
        else:
            assert 64 <= t.m == t.n == t.k <= 4096
    for r in range(64):
        arr = [t.arrival_s for t in w.tasks if t.rank == r]
        assert all(b > a for a, b in zip(arr, arr[1:]))
    w2 = synth.stress_mix(ranks=64, per_rank=32)
    assert [(t.n, t.m, t.arrival_s) for t in w.tasks] == [(t.n, t.m, t.arrival_s) for t in w2.tasks]
