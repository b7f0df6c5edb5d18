/*
 * A plain C client of the C ABI (include/gvm.h): no Python, no PyTorch. It
 * owns its device memory (CUDA runtime), starts a manager in barrier mode,
 * attaches two ranks, submits a vector add on rank 0 and a matrix multiply on
 * rank 1 (host mode, page-locked buffers), flushes, syncs both, and writes the
 * results for the test that drives it to compare with the CPU oracle.
 *
 *   gvm_c_client <inputs> <outputs>
 *   inputs:  int64 n, int32 m, k, nn, float a[n], b[n], A[m*k], B[k*nn]
 *   outputs: float c[n], C[m*nn]
 * Exit status 0 on success; a message on stderr otherwise.
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "gvm.h"

#define FAIL(...)                     \
  do {                                \
    fprintf(stderr, __VA_ARGS__);     \
    fputc('\n', stderr);              \
    return 1;                         \
  } while (0)
#define GVM(call)                                                                      \
  do {                                                                                 \
    int rc_ = (call);                                                                  \
    if (rc_ != GVM_OK) FAIL("%s failed: %d (%s)", #call, rc_, gvm_strerror(rc_));      \
  } while (0)
#define CUDA(call)                                                                     \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) FAIL("%s failed: %s", #call, cudaGetErrorString(e_));       \
  } while (0)

static int read_all(FILE* f, void* p, size_t bytes) { return fread(p, 1, bytes, f) == bytes ? 0 : 1; }

int main(int argc, char** argv) {
  if (argc != 3) FAIL("usage: %s <inputs> <outputs>", argv[0]);
  FILE* fi = fopen(argv[1], "rb");
  if (!fi) FAIL("cannot open %s", argv[1]);
  int64_t n = 0;
  int32_t m = 0, k = 0, nn = 0;
  if (read_all(fi, &n, 8) || read_all(fi, &m, 4) || read_all(fi, &k, 4) || read_all(fi, &nn, 4))
    FAIL("short header");

  CUDA(cudaSetDevice(0));
  float *a, *b, *c, *A, *B, *C;
  CUDA(cudaHostAlloc((void**)&a, 4 * (size_t)n, cudaHostAllocDefault));
  CUDA(cudaHostAlloc((void**)&b, 4 * (size_t)n, cudaHostAllocDefault));
  CUDA(cudaHostAlloc((void**)&c, 4 * (size_t)n, cudaHostAllocDefault));
  CUDA(cudaHostAlloc((void**)&A, 4 * (size_t)m * k, cudaHostAllocDefault));
  CUDA(cudaHostAlloc((void**)&B, 4 * (size_t)k * nn, cudaHostAllocDefault));
  CUDA(cudaHostAlloc((void**)&C, 4 * (size_t)m * nn, cudaHostAllocDefault));
  if (read_all(fi, a, 4 * (size_t)n) || read_all(fi, b, 4 * (size_t)n) || read_all(fi, A, 4 * (size_t)m * k) ||
      read_all(fi, B, 4 * (size_t)k * nn))
    FAIL("short inputs");
  fclose(fi);

  gvm_config cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.max_ranks = 2;
  cfg.ring_depth = 8;
  cfg.mode = GVM_MODE_BARRIER;
  cfg.sgemm_path = GVM_SGEMM_SPLIT3;
  const uint64_t slice = 64ull << 20;
  const uint64_t ctrl_bytes = gvm_ctrl_bytes(&cfg);
  if (ctrl_bytes == 0) FAIL("gvm_ctrl_bytes refused the configuration");
  void *arena, *ctrl;
  CUDA(cudaMalloc(&arena, 2 * slice));  /* 256-byte aligned */
  CUDA(cudaMalloc(&ctrl, ctrl_bytes));
  cfg.arena = arena;
  cfg.arena_bytes = 2 * slice;
  cfg.ctrl = ctrl;
  cfg.ctrl_bytes = ctrl_bytes;

  gvm_ctx* ctx = NULL;
  GVM(gvm_init(&cfg, &ctx));
  gvm_rank *r0 = NULL, *r1 = NULL;
  GVM(gvm_attach(ctx, 0, &r0));
  GVM(gvm_attach(ctx, 1, &r1));

  gvm_task t0, t1;
  memset(&t0, 0, sizeof(t0));
  memset(&t1, 0, sizeof(t1));
  t0.type = GVM_TASK_VADD;
  t0.n = n;
  t0.a = a;
  t0.b = b;
  t0.c = c;
  t1.type = GVM_TASK_SGEMM;
  t1.m = m;
  t1.k = k;
  t1.n = nn;
  t1.a = A;
  t1.b = B;
  t1.c = C;
  uint64_t s0 = 0, s1 = 0;
  GVM(gvm_submit(r0, &t0, &s0));
  GVM(gvm_submit(r1, &t1, &s1));
  GVM(gvm_flush(ctx)); /* the request barrier */
  GVM(gvm_sync(r0, s0));
  GVM(gvm_sync(r1, s1));
  if (gvm_poll(r0, s0) != 1 || gvm_poll(r1, s1) != 1) FAIL("poll after sync");
  GVM(gvm_detach(r0));
  GVM(gvm_detach(r1));
  GVM(gvm_shutdown(ctx));

  FILE* fo = fopen(argv[2], "wb");
  if (!fo) FAIL("cannot open %s", argv[2]);
  if (fwrite(c, 4, (size_t)n, fo) != (size_t)n || fwrite(C, 4, (size_t)m * nn, fo) != (size_t)m * nn)
    FAIL("short write");
  fclose(fo);
  CUDA(cudaFree(arena));
  CUDA(cudaFree(ctrl));
  CUDA(cudaFreeHost(a));
  CUDA(cudaFreeHost(b));
  CUDA(cudaFreeHost(c));
  CUDA(cudaFreeHost(A));
  CUDA(cudaFreeHost(B));
  CUDA(cudaFreeHost(C));
  return 0;
}
