/*
 * CPU oracle for the GPU-sharing hot path: test infrastructure only.
 *
 * Plain, slow, obviously correct restatements of what each shared-GPU task
 * computes. Only tests, the smoke check and the bench's CPU-baseline leg may
 * call this library; the product path never links or loads it.
 *
 * The paper (Li, Narayana, El-Ghazawi, "Efficient Resource Sharing Through
 * GPU Virtualization on Accelerated HPC Systems", Section 6, Table 2) runs
 * two task kernels that this build keeps: a single-precision vector addition
 * and a single-precision matrix multiplication. Sharing the GPU changes only
 * the timing of a task (Section 4.2.2, Section 5), so each task's result is
 * defined by the task alone:
 *
 *   vector add (Table 2, "VecAdd"): c[i] = fl32(a[i] + b[i]), one IEEE-754
 *     binary32 addition, round to nearest even, subnormals kept.
 *   vector multiply (Table 2, "VecMult", 15 iterations there): c[i] =
 *     fl32(...fl32(fl32(a[i] * b[i]) * b[i]) ... * b[i]) with `iters`
 *     binary32 multiplications in turn, each rounded to nearest even.
 *   matrix multiply (Table 2, "MM"; Section 6 calls it single precision):
 *     C[i][j] = sum_k A[i][k] * B[k][j], row-major A (M x K), B (K x N),
 *     C (M x N), computed here in binary64 with k = 0 .. K-1 in order.
 *
 * Build with -O2 -ffp-contract=off so that no multiply-add is fused and the
 * binary64 sum follows the written order.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

/* Vector add: one binary32 addition per element (Table 2, VecAdd). */
void oracle_vadd_f32(const float* a, const float* b, float* c, int64_t n) {
  for (int64_t i = 0; i < n; ++i) c[i] = a[i] + b[i];
}

/*
 * Vector multiply (Table 2, VecMult): the element is multiplied by b[i]
 * `iters` times in binary32, one rounding per product.
 */
void oracle_vmul_f32(const float* a, const float* b, float* c, int64_t n, int32_t iters) {
  for (int64_t i = 0; i < n; ++i) {
    float z = a[i];
    for (int32_t t = 0; t < iters; ++t) z = z * b[i];
    c[i] = z;
  }
}

/*
 * Matrix multiply in binary64 (Table 2, MM). Loop order i, k, j: for every
 * output element the products are added for k = 0, 1, ..., K-1 in turn.
 */
void oracle_sgemm_f64(const float* A, const float* B, double* C, int64_t M, int64_t N,
                      int64_t K) {
  for (int64_t i = 0; i < M; ++i) {
    double* c = C + i * N;
    for (int64_t j = 0; j < N; ++j) c[j] = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      const double a = (double)A[i * K + k];
      const float* b = B + k * N;
      for (int64_t j = 0; j < N; ++j) c[j] += a * (double)b[j];
    }
  }
}

/*
 * Relative Frobenius error ||C - R||_F / ||R||_F of a binary32 result C
 * against the binary64 oracle R, both norms accumulated in binary64.
 * Returns 0 when both are zero and +inf when only R is zero.
 */
double oracle_rel_fro_err(const float* C, const double* R, int64_t count) {
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < count; ++i) {
    const double d = (double)C[i] - R[i];
    num += d * d;
    den += R[i] * R[i];
  }
  if (den == 0.0) return num == 0.0 ? 0.0 : INFINITY;
  return sqrt(num) / sqrt(den);
}
