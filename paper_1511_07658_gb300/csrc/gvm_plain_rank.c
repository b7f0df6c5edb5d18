/* One rank of the plain, non-virtualized form (Section 4.1, Eq. 1): a
 * process of its own with its own CUDA context, running its tasks one after
 * another on the default stream with synchronous copies, through the same
 * task kernels the manager runs (gvm_sgemm_f32). Sixteen of these side by
 * side are the conventional sharing the virtualization manager replaces; the
 * benchmark starts them and compares their turnaround with the shared form.
 *
 * Usage: gvm_plain_rank TASKS M N K INFILE OUTFILE CORE INIT PHASE...
 *   INFILE   TASKS x (A (M x K) then B (K x N)) binary32, row-major
 *   OUTFILE  C (M x N) of the last task of phase i is written to OUTFILE.i
 *   CORE     host core the process pins itself to (-1: none), as the paper
 *            pins each process to a core
 *   INIT     "before": the context, the device buffers and the page-locking
 *            of the host buffers are made before the first start signal;
 *            "timed": after it, inside the first phase's timed region
 *            (T_init of Eq. 1; the first phase must then copy)
 *   PHASE    PATH:MODE, run in order, each on its own start signal:
 *            PATH  GVM_SGEMM_* path number (0 = FMA, 2 = split3 fused)
 *            MODE  resident  operands copied to the device before the
 *                            first start; per task kernel + synchronize
 *                  copy      per task: copy A and B in, kernel, copy C out
 *                            (synchronous)
 *
 * Protocol on stdin/stdout: the process reads its inputs, initialises
 * (INIT = before), prints "ready CTX ALLOC PIN" (ns spent creating the
 * context, allocating device memory and page-locking host memory), then per
 * phase waits for one byte on stdin, runs, writes OUTFILE.i and then prints
 * "T0 T1 T_INIT RC" (CLOCK_MONOTONIC ns at the start and end of the timed
 * region, the ns of initialisation inside it, status 0 = ok).
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

enum { MODE_RESIDENT = 0, MODE_COPY = 1 };

struct Rank {
  int tasks, m, n, k;
  size_t a_elems, b_elems, c_elems;
  float* host_in;   /* tasks x (A, B), page-locked at init */
  float* host_out;  /* tasks x C, page-locked at init */
  float* dev_in;    /* tasks x (A, B) */
  float* dev_out;   /* tasks x C */
  uint64_t t_ctx, t_alloc, t_pin;
};

/* Context, device buffers, page-locked host buffers: the per-process
 * initialisation the plain form pays and the manager pays once. */
static int init_gpu(struct Rank* r) {
  const uint64_t t0 = now_ns();
  if (cudaSetDevice(0) != cudaSuccess) return 1;
  if (cudaFree(0) != cudaSuccess) return 2;
  const uint64_t t1 = now_ns();
  const size_t per_in = r->a_elems + r->b_elems;
  if (cudaMalloc((void**)&r->dev_in, (size_t)r->tasks * per_in * sizeof(float)) != cudaSuccess) return 3;
  if (cudaMalloc((void**)&r->dev_out, (size_t)r->tasks * r->c_elems * sizeof(float)) != cudaSuccess) return 4;
  const uint64_t t2 = now_ns();
  if (cudaHostRegister(r->host_in, (size_t)r->tasks * per_in * sizeof(float), cudaHostRegisterDefault) !=
      cudaSuccess)
    return 5;
  if (cudaHostRegister(r->host_out, (size_t)r->tasks * r->c_elems * sizeof(float), cudaHostRegisterDefault) !=
      cudaSuccess)
    return 6;
  if (cudaDeviceSynchronize() != cudaSuccess) return 7;
  const uint64_t t3 = now_ns();
  r->t_ctx = t1 - t0;
  r->t_alloc = t2 - t1;
  r->t_pin = t3 - t2;
  return 0;
}

/* One phase: every task in order; the last result is left in host_out. */
static int run_tasks(struct Rank* r, int path, int mode) {
  const size_t per_in = r->a_elems + r->b_elems;
  for (int t = 0; t < r->tasks; ++t) {
    const float* hA = r->host_in + (size_t)t * per_in;
    float* hC = r->host_out + (size_t)t * r->c_elems;
    float *dA, *dB, *dC;
    if (mode == MODE_RESIDENT) {
      dA = r->dev_in + (size_t)t * per_in;
      dB = dA + r->a_elems;
      dC = r->dev_out + (size_t)t * r->c_elems;
    } else {
      dA = r->dev_in;
      dB = dA + r->a_elems;
      dC = r->dev_out;
      if (cudaMemcpy(dA, hA, per_in * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return 10;
    }
    const int rc = gvm_sgemm_f32(dA, dB, dC, r->m, r->n, r->k, path, NULL, 0, NULL);
    if (rc != GVM_OK) return 100 - rc;
    if (mode == MODE_RESIDENT) {
      if (cudaDeviceSynchronize() != cudaSuccess) return 11;
    } else if (cudaMemcpy(hC, dC, r->c_elems * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
      return 12;
    }
  }
  if (mode == MODE_RESIDENT) {
    const size_t last = (size_t)(r->tasks - 1) * r->c_elems;
    if (cudaMemcpy(r->host_out + last, r->dev_out + last, r->c_elems * sizeof(float), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return 13;
  }
  return 0;
}

int main(int argc, char** argv) {
  if (argc < 10) {
    fprintf(stderr, "usage: %s TASKS M N K INFILE OUTFILE CORE INIT PHASE...\n", argv[0]);
    return 2;
  }
  const int core = atoi(argv[7]);
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
  if (r.tasks <= 0 || r.m <= 0 || r.n <= 0 || r.k <= 0) return 2;
  const int init_timed = !strcmp(argv[8], "timed");
  if (!init_timed && strcmp(argv[8], "before")) return 2;
  const int nphases = argc - 9;
  int paths[16], modes[16];
  if (nphases > 16) return 2;
  for (int i = 0; i < nphases; ++i) {
    const char* ph = argv[9 + i];
    const char* colon = strchr(ph, ':');
    if (!colon) return 2;
    paths[i] = atoi(ph);
    if (!strcmp(colon + 1, "resident")) modes[i] = MODE_RESIDENT;
    else if (!strcmp(colon + 1, "copy")) modes[i] = MODE_COPY;
    else return 2;
    if (init_timed && modes[i] == MODE_RESIDENT) return 2;
  }
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
  FILE* f = fopen(argv[5], "rb");
  if (!f || fread(r.host_in, 1, in_bytes, f) != in_bytes) return 4;
  fclose(f);
  memset(r.host_out, 0, out_bytes);

  int rc = 0;
  if (!init_timed) {
    rc = init_gpu(&r);
    if (!rc && cudaMemcpy(r.dev_in, r.host_in, in_bytes, cudaMemcpyHostToDevice) != cudaSuccess) rc = 20;
  }
  printf("ready %llu %llu %llu\n", (unsigned long long)r.t_ctx, (unsigned long long)r.t_alloc,
         (unsigned long long)r.t_pin);
  fflush(stdout);
  char name[4096];
  for (int i = 0; i < nphases; ++i) {
    char go = 0;
    if (fread(&go, 1, 1, stdin) != 1) return 5;
    const uint64_t t0 = now_ns();
    uint64_t t_init = 0;
    if (!rc && init_timed && i == 0) {
      rc = init_gpu(&r);
      t_init = now_ns() - t0;
    }
    if (!rc) rc = run_tasks(&r, paths[i], modes[i]);
    const uint64_t t1 = now_ns();
    // The result file is complete before the line that reports the phase.
    snprintf(name, sizeof(name), "%s.%d", argv[6], i);
    FILE* o = fopen(name, "wb");
    if (!o) return 6;
    const size_t last = (size_t)(r.tasks - 1) * r.c_elems;
    if (fwrite(r.host_out + last, sizeof(float), r.c_elems, o) != r.c_elems) rc = rc ? rc : 30;
    if (fclose(o) != 0) rc = rc ? rc : 31;
    printf("%llu %llu %llu %d\n", (unsigned long long)t0, (unsigned long long)t1, (unsigned long long)t_init, rc);
    fflush(stdout);
  }
  return rc ? 1 : 0;
}
