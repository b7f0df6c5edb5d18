/* One rank of the plain, non-virtualized form (Section 4.1, Eq. 1): a
 * process of its own with its own CUDA context, running its tasks one after
 * another on the default stream with synchronous copies, through the same
 * task kernels the manager runs (gvm_sgemm_f32). Sixteen of these side by
 * side are the conventional sharing the virtualization manager replaces; the
 * benchmark starts them and compares their turnaround with the shared form.
 *
 * Usage: gvm_plain_rank TASKS M N K PATH MODE INFILE OUTFILE CORE
 *   PATH     GVM_SGEMM_* path number (0 = FMA, 2 = split3 fused)
 *   MODE     resident   operands copied to the device before the start;
 *                       the timed loop is kernel + synchronize per task
 *            copy       per task: copy A and B in, kernel, copy C out
 *                       (synchronous), context made before the start
 *            copy_init  as copy, but the context, the device buffers and
 *                       the page-locking of the host buffers are made
 *                       inside the timed region (T_init of Eq. 1)
 *   INFILE   TASKS x (A (M x K) then B (K x N)) binary32, row-major
 *   OUTFILE  C (M x N) of the last task is written here
 *   CORE     host core the process pins itself to (-1: none), as the paper
 *            pins each process to a core
 *
 * Protocol on stdin/stdout: the process reads its inputs and (except in
 * copy_init) initialises, prints "ready", waits for one byte on stdin, runs,
 * then prints one line "t0 t1 t_init rc" (CLOCK_MONOTONIC ns for the start
 * and end of the timed region, T_init in ns, GVM/CUDA status 0 = ok).
 */
#define _GNU_SOURCE
#include <cuda_runtime.h>
#include <sched.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "gvm.h"

static uint64_t now_ns(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

enum { MODE_RESIDENT = 0, MODE_COPY = 1, MODE_COPY_INIT = 2 };

struct Rank {
  int tasks, m, n, k, path, mode;
  size_t a_elems, b_elems, c_elems;
  float* host_in;   /* tasks x (A, B), page-locked after init */
  float* host_out;  /* tasks x C, page-locked after init */
  float* dev_in;    /* resident: tasks x (A, B); copy: one (A, B) */
  float* dev_out;   /* resident: tasks x C; copy: one C */
};

/* Context, device buffers, page-locked host buffers: the per-process
 * initialisation the plain form pays and the manager pays once. */
static int init_gpu(struct Rank* r) {
  if (cudaSetDevice(0) != cudaSuccess) return 1;
  if (cudaFree(0) != cudaSuccess) return 2;
  const size_t per_in = r->a_elems + r->b_elems;
  const size_t n_in = r->mode == MODE_RESIDENT ? (size_t)r->tasks * per_in : per_in;
  const size_t n_out = r->mode == MODE_RESIDENT ? (size_t)r->tasks * r->c_elems : r->c_elems;
  if (cudaMalloc((void**)&r->dev_in, n_in * sizeof(float)) != cudaSuccess) return 3;
  if (cudaMalloc((void**)&r->dev_out, n_out * sizeof(float)) != cudaSuccess) return 4;
  if (cudaHostRegister(r->host_in, (size_t)r->tasks * per_in * sizeof(float), cudaHostRegisterDefault) !=
      cudaSuccess)
    return 5;
  if (cudaHostRegister(r->host_out, (size_t)r->tasks * r->c_elems * sizeof(float), cudaHostRegisterDefault) !=
      cudaSuccess)
    return 6;
  if (cudaDeviceSynchronize() != cudaSuccess) return 7;
  return 0;
}

static int run_tasks(struct Rank* r) {
  const size_t per_in = r->a_elems + r->b_elems;
  for (int t = 0; t < r->tasks; ++t) {
    const float* hA = r->host_in + (size_t)t * per_in;
    float* hC = r->host_out + (size_t)t * r->c_elems;
    float *dA, *dB, *dC;
    if (r->mode == MODE_RESIDENT) {
      dA = r->dev_in + (size_t)t * per_in;
      dB = dA + r->a_elems;
      dC = r->dev_out + (size_t)t * r->c_elems;
    } else {
      dA = r->dev_in;
      dB = dA + r->a_elems;
      dC = r->dev_out;
      if (cudaMemcpy(dA, hA, per_in * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return 10;
    }
    const int rc = gvm_sgemm_f32(dA, dB, dC, r->m, r->n, r->k, r->path, NULL, 0, NULL);
    if (rc != GVM_OK) return 100 - rc;
    if (r->mode == MODE_RESIDENT) {
      if (cudaDeviceSynchronize() != cudaSuccess) return 11;
    } else if (cudaMemcpy(hC, dC, r->c_elems * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
      return 12;
    }
  }
  if (r->mode == MODE_RESIDENT) {
    const size_t last = (size_t)(r->tasks - 1) * r->c_elems;
    if (cudaMemcpy(r->host_out + last, r->dev_out + last, r->c_elems * sizeof(float), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return 13;
  }
  return 0;
}

int main(int argc, char** argv) {
  if (argc != 10) {
    fprintf(stderr, "usage: %s TASKS M N K PATH MODE INFILE OUTFILE CORE\n", argv[0]);
    return 2;
  }
  const int core = atoi(argv[9]);
  if (core >= 0) {
    cpu_set_t set;
    CPU_ZERO(&set);
    CPU_SET(core, &set);
    if (sched_setaffinity(0, sizeof(set), &set) != 0) return 2;
  }
  struct Rank r;
  memset(&r, 0, sizeof(r));
  r.tasks = atoi(argv[1]);
  r.m = atoi(argv[2]);
  r.n = atoi(argv[3]);
  r.k = atoi(argv[4]);
  r.path = atoi(argv[5]);
  if (!strcmp(argv[6], "resident")) r.mode = MODE_RESIDENT;
  else if (!strcmp(argv[6], "copy")) r.mode = MODE_COPY;
  else if (!strcmp(argv[6], "copy_init")) r.mode = MODE_COPY_INIT;
  else return 2;
  if (r.tasks <= 0 || r.m <= 0 || r.n <= 0 || r.k <= 0) return 2;
  r.a_elems = (size_t)r.m * r.k;
  r.b_elems = (size_t)r.k * r.n;
  r.c_elems = (size_t)r.m * r.n;
  const size_t in_bytes = (size_t)r.tasks * (r.a_elems + r.b_elems) * sizeof(float);
  const size_t out_bytes = (size_t)r.tasks * r.c_elems * sizeof(float);
  void* pin = NULL;
  void* pout = NULL;
  if (posix_memalign(&pin, 4096, in_bytes) || posix_memalign(&pout, 4096, out_bytes)) return 3;
  r.host_in = (float*)pin;
  r.host_out = (float*)pout;
  FILE* f = fopen(argv[7], "rb");
  if (!f || fread(r.host_in, 1, in_bytes, f) != in_bytes) return 4;
  fclose(f);
  memset(r.host_out, 0, out_bytes);

  uint64_t t_init = 0;
  int rc = 0;
  if (r.mode != MODE_COPY_INIT) {
    const uint64_t i0 = now_ns();
    rc = init_gpu(&r);
    t_init = now_ns() - i0;
    if (!rc && r.mode == MODE_RESIDENT &&
        cudaMemcpy(r.dev_in, r.host_in, in_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      rc = 20;
  }
  printf("ready\n");
  fflush(stdout);
  char go = 0;
  if (fread(&go, 1, 1, stdin) != 1) return 5;
  const uint64_t t0 = now_ns();
  if (!rc && r.mode == MODE_COPY_INIT) {
    rc = init_gpu(&r);
    t_init = now_ns() - t0;
  }
  if (!rc) rc = run_tasks(&r);
  const uint64_t t1 = now_ns();
  printf("%llu %llu %llu %d\n", (unsigned long long)t0, (unsigned long long)t1, (unsigned long long)t_init, rc);
  fflush(stdout);
  FILE* o = fopen(argv[8], "wb");
  if (!o) return 6;
  const size_t last = (size_t)(r.tasks - 1) * r.c_elems;
  fwrite(r.host_out + last, sizeof(float), r.c_elems, o);
  fclose(o);
  return rc ? 1 : 0;
}
