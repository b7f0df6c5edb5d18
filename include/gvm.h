/*
 * gvm.h -- C ABI of the GB300 GPU virtualization manager.
 *
 * The method (Li, Narayana, El-Ghazawi, "Efficient Resource Sharing Through
 * GPU Virtualization on Accelerated High Performance Computing Systems"):
 * many SPMD processes share one GPU through a single virtualization manager
 * that owns the only GPU context, gives each process a virtual GPU with its
 * own memory objects and stream, and runs every process's task -- an input
 * copy, a data-parallel kernel, an output copy -- concurrently with the
 * others (Section 4.2.2, Section 5). This header is that manager's boundary.
 *
 * Mapping of the paper's API routines (Section 5):
 *   REQ()          -> gvm_attach   (get a virtual GPU: ring, arena slice, streams)
 *   SND() + STR()  -> gvm_submit   (hand over the input, start the kernel)
 *   STP() + RCV()  -> gvm_sync     (wait for the result to be back in host memory)
 *   RLS()          -> gvm_detach   (release the virtual GPU)
 *   request barrier-> gvm_flush    (barrier mode: drain everything submitted so far)
 *
 * Conventions:
 *   - Every entry point returns GVM_OK (0) or a negative GVM_E* code; no C++
 *     exception crosses this boundary.
 *   - The library owns no device memory: the caller passes device memory
 *     (arena, control block) and stream handles; the library never calls
 *     cudaMalloc. It allocates pinned host memory for the task rings only.
 *   - A gvm_rank handle is used by one host thread at a time; different ranks
 *     may be driven concurrently from different threads.
 *   - Stream arguments are cudaStream_t values passed as void*.
 */
#ifndef GVM_H
#define GVM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GVM_API __attribute__((visibility("default")))
#else
#define GVM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define GVM_OK 0
#define GVM_EINVAL (-1)     /* bad argument, shape or offset */
#define GVM_EBUSY (-2)      /* rank already attached */
#define GVM_EAGAIN (-3)     /* ring or staging space full right now; retry after gvm_sync */
#define GVM_ENOMEM (-4)     /* the task can never fit its rank's staging space or the cap */
#define GVM_ETIMEDOUT (-5)  /* a bounded wait ran out (host or device side) */
#define GVM_EDEVICE (-6)    /* a CUDA call failed or the device reported an error status */
#define GVM_ECANCELED (-7)  /* the manager shut down before the task completed */
#define GVM_ESTATE (-8)     /* call not valid in the current state (e.g. not attached) */
#define GVM_ENODEV (-9)     /* no usable CUDA device */

/* ---- task types (Section 6, Table 2) ------------------------------------ */
#define GVM_TASK_VADD 1   /* c[i] = a[i] + b[i], binary32, n elements */
#define GVM_TASK_SGEMM 2  /* C = A B, binary32, row-major A (m x k), B (k x n), C (m x n) */
#define GVM_TASK_VMUL 3   /* c[i] = a[i] * b[i] * ... * b[i] with k binary32 products, each
                             rounded to nearest (Table 2, VecMul: the I/O-intensive task of
                             the model validation, 15 iterations), n elements */

/* ---- task flags --------------------------------------------------------- */
#define GVM_TASK_RESIDENT 1 /* a_off/b_off/c_off address the rank's resident region;
                               no host copies (inputs already on the device) */

/* ---- SGEMM arithmetic --------------------------------------------------- */
#define GVM_SGEMM_FMA 0    /* binary32 fused multiply-add on the CUDA cores */
#define GVM_SGEMM_SPLIT3 1 /* A = Ah + Al, B = Bh + Bl in bf16; C = AhBh + AhBl + AlBh on
                              tcgen05 tensor cores with binary32 accumulation in TMEM.
                              The manager splits while staging operands into shared
                              memory (no scratch); gvm_sgemm_f32 runs a split pre-pass
                              into caller scratch, then TMA-fed GEMM tiles */
#define GVM_SGEMM_SPLIT3_FUSED 2 /* gvm_sgemm_f32 only: the manager's form of split3 (split
                              during staging, no scratch); bit-identical to
                              GVM_SGEMM_SPLIT3 */
/* 3 is not used (it named a removed form); gvm_sgemm_f32 refuses it. */
#define GVM_SGEMM_SPLIT3_WIDE 4 /* split during staging on 256 x 256 tiles of one CTA (the
                              two 128-row halves share each B stage; one accumulator);
                              bit-identical to GVM_SGEMM_SPLIT3. Also a manager path */
#define GVM_SGEMM_SPLIT3_TMA 5 /* manager path only: 128 x 256 tiles whose binary32 A and B
                              arrive by TMA boxes (a tensor map of each per task, where A
                              and B are 16-byte aligned with row pitches of 16-byte
                              multiples; other tasks are loaded by the converting warps)
                              and are split in place; bit-identical to GVM_SGEMM_SPLIT3 */

/* ---- manager modes ------------------------------------------------------ */
#define GVM_MODE_BARRIER 0    /* Section 5 request barrier: gvm_flush runs the scheduler
                                 until every task submitted before it has completed */
#define GVM_MODE_CONTINUOUS 1 /* the scheduler is launched by gvm_init, stays resident
                                 and takes tasks as they arrive, until gvm_shutdown. It
                                 holds every SM meanwhile (idle CTAs sleep between polls),
                                 so a device-wide synchronisation in the process
                                 (cudaDeviceSynchronize, cudaFree, cudaFreeHost) waits
                                 until gvm_shutdown */
/* The paper's own mechanism (Sections 4.2.1 and 5): no persistent scheduler.
   gvm_flush is the request barrier; it issues every task submitted before it
   on its rank's stream (the input stream of gvm_stream) as separate copies of
   each operand and one launch of the task's kernel (gvm_vadd_f32,
   gvm_vmul_f32, or gvm_sgemm_f32 on the manager's SGEMM path), followed by the
   completion word. Submission only validates and stages. */
#define GVM_MODE_PS1 2 /* programming style 1: all ranks' input copies, then all
                          kernels, then all output copies (Eq. 2 / Eq. 4) */
#define GVM_MODE_PS2 3 /* programming style 2: rank by rank, each task's input,
                          kernel and output in turn (Eq. 3 / Eqs. 5-7) */

#define GVM_MAX_RANKS 1024

typedef struct gvm_config {
  int32_t max_ranks;      /* ranks that may attach: 1 .. GVM_MAX_RANKS */
  int32_t ring_depth;     /* task descriptors per rank; power of two, 2 .. 4096 */
  int32_t mode;           /* GVM_MODE_BARRIER, GVM_MODE_CONTINUOUS, GVM_MODE_PS1 or
                             GVM_MODE_PS2 */
  int32_t sgemm_path;     /* GVM_SGEMM_FMA, GVM_SGEMM_SPLIT3, GVM_SGEMM_SPLIT3_WIDE or
                             GVM_SGEMM_SPLIT3_TMA */
  void* arena;            /* caller-owned device memory, 256-byte aligned. Split into
                             max_ranks equal slices (Section 5: one memory object per
                             process, so data of different processes coexist safely) */
  uint64_t arena_bytes;
  uint64_t resident_bytes; /* bytes at the start of each slice addressed by the offsets
                              of GVM_TASK_RESIDENT tasks; the rest of the slice is the
                              rank's staging ring (copied inputs and outputs) */
  void* ctrl;             /* caller-owned device memory for control words and the
                             device task table, >= gvm_ctrl_bytes(cfg), 256-aligned */
  uint64_t ctrl_bytes;
  void* sched_stream;     /* cudaStream_t on which the scheduler kernel is launched, or
                             NULL: the manager creates a non-blocking stream */
  void* const* copy_streams; /* 2*max_ranks distinct cudaStream_t: [2r] carries rank r's
                                input copies, [2r+1] its output copies (Section 4.2.1:
                                one stream per process), or NULL: the manager creates
                                them. Streams it creates are destroyed by gvm_shutdown;
                                see gvm_stream */
  uint64_t admission_cap_bytes; /* cap on staging bytes held by admitted, unfinished tasks
                                   across all ranks; 0 = only the slices bound it */
  uint64_t wait_timeout_ns; /* bound on each device-side dependency wait and on each
                               host wait in gvm_sync / gvm_wait_idle; 0 = 10 s */
  uint64_t idle_poll_ns;    /* sleep of an idle scheduler CTA between polls of the
                               rings; 0 = 1000 ns */
  int32_t grid_ctas;        /* scheduler CTAs; 0 = one per SM */
  int32_t ingest_quantum;   /* tasks taken from one rank per ingest pass; 0 = 4 */
  uint64_t copy_run_bytes;  /* host-mode copies of one batch that are adjacent on both
                               sides are merged up to this many bytes; 0 = 16 MiB */
  int64_t vadd_tile;        /* elements per vector-add tile (rounded to 1024); 0 = per
                               task: n / scheduler CTAs, within 16 Ki .. 1 Mi */
  int32_t direct_output;    /* barrier and continuous modes, host-mode tasks: 0 = the
                               result is staged in the rank's slice and copied to c by the
                               rank's output stream (Section 5's data path); 1 = the
                               scheduler writes it straight into c through the buffer's
                               device mapping (page-locked memory the GPU can address;
                               a buffer without one uses the staged path), so outputs
                               take no staging and no copy */
  int32_t l2_prefetch;      /* split3: 1 = the claiming warp asks L2 for each task's operands
                               (bulk prefetch, a few tiles ahead; a hint, no result depends
                               on it); 0 = off */
  int32_t copy_streams_max; /* copy_streams NULL: at most this many copy streams are created
                               (0 = 31, which with the scheduler's stream fills the 32
                               hardware queues of CUDA_DEVICE_MAX_CONNECTIONS=32); while
                               2 x max_ranks exceeds it, ranks share input streams (r % n_in)
                               and output streams (r % n_out), n_in + n_out <= the limit */
  int32_t copy_in_streams;  /* copy_streams NULL: input copy streams to create (ranks share
                               them round robin, r % n), the rest of copy_streams_max going
                               to output streams; 0 = split the limit evenly. One input
                               stream lands a step's inputs in submission order, all of a
                               step before the next step's */
} gvm_config;

typedef struct gvm_task {
  int32_t type;   /* GVM_TASK_VADD, GVM_TASK_SGEMM or GVM_TASK_VMUL */
  int32_t flags;  /* 0 or GVM_TASK_RESIDENT */
  int64_t n;      /* VADD, VMUL: element count (>= 0). SGEMM: columns of B and C (>= 1) */
  int32_t m;      /* SGEMM: rows of A and C (>= 1) */
  int32_t k;      /* SGEMM: columns of A, rows of B (>= 1). VMUL: products per element
                     (1 .. 1024) */
  /* host mode (flags without GVM_TASK_RESIDENT): host buffers, caller-owned,
     valid and untouched until gvm_sync returns for this task. Page-locked
     buffers are copied asynchronously; pageable ones are accepted too (the
     driver stages their input copies, and a pageable result is copied out by
     the rank's gvm_sync / gvm_poll once the task has completed). Device or
     managed memory is refused (GVM_EINVAL): a rank reaches the GPU only
     through the manager's copies.
     VADD, VMUL: a, b, c hold n floats. SGEMM: a = A (m*k), b = B (k*n), c = C (m*n). */
  const void* a;
  const void* b;
  void* c;
  /* resident mode: byte offsets into the rank's resident region, 16-byte aligned
     for SGEMM and 4-byte aligned for VADD and VMUL; operands must lie inside the
     region. */
  uint64_t a_off;
  uint64_t b_off;
  uint64_t c_off;
} gvm_task;

typedef struct gvm_stats {
  uint64_t submitted;      /* tasks accepted by gvm_submit */
  uint64_t completed;      /* tasks observed complete by gvm_sync / gvm_poll */
  uint64_t launches;       /* scheduler kernel launches */
  uint64_t staged_bytes;   /* staging bytes currently held by unfinished tasks */
  uint64_t staged_peak;    /* high-water mark of staged_bytes */
  uint64_t h2d_bytes;      /* bytes copied host to device by the manager */
  uint64_t d2h_bytes;      /* bytes copied device to host by the manager */
  uint32_t device_status;  /* last error status word written by the scheduler (0 = ok) */
  uint32_t device_where;   /* which wait or check set device_status */
  uint64_t launch_start_ns;     /* last scheduler launch that exited: first CTA start, */
  uint64_t launch_last_done_ns; /* its last task completion and its last CTA exit */
  uint64_t launch_exit_ns;      /* (device %globaltimer, ns; 0 before any exit) */
  uint64_t launch_phase[12];    /* that launch's CTA time per phase, summed over CTAs (ns):
                                   [0] finding work (claims, ingest, idle polling),
                                   [1] ingest passes that published work, [2] split3:
                                   staging warps waiting for a free stage, [3] GEMM tiles
                                   (split3: staging warps' time incl. [8]), [4] split3: MMA
                                   warp waiting for a staged k-step, [5] vector-add tiles;
                                   counts: [6] tiles run, [7] ingest passes that published
                                   work; [8] split3: draining accumulators into C;
                                   [9..11] 0 */
} gvm_stats;

typedef struct gvm_ctx gvm_ctx;
typedef struct gvm_rank gvm_rank;

/* Device bytes the control block needs for cfg (depends on max_ranks and
   ring_depth only). Returns 0 for an invalid cfg. */
GVM_API uint64_t gvm_ctrl_bytes(const gvm_config* cfg);

/* Creates the manager (Section 5: the GVM initialises every resource once,
   which hides T_init, Section 4.2.3). Checks cfg, zeroes the control block on
   sched_stream, allocates the pinned rings and, in continuous mode, launches
   the scheduler. *out receives the handle. Errors: GVM_EINVAL (cfg),
   GVM_ENODEV, GVM_EDEVICE, GVM_ENOMEM (host rings). */
GVM_API int gvm_init(const gvm_config* cfg, gvm_ctx** out);

/* REQ(): attaches rank 0 <= rank < max_ranks and returns its handle.
   GVM_EBUSY if attached already, GVM_EINVAL if out of range. */
GVM_API int gvm_attach(gvm_ctx* ctx, int32_t rank, gvm_rank** out);

/* SND() + STR(): admits one task and returns at once. Host mode enqueues the
   input copies on the rank's input stream, then a ready flag; the output copy
   waits on the task's done flag on the rank's output stream. Resident mode
   enqueues nothing. The task then runs when the scheduler takes it from the
   ring. *seq_out receives its sequence number (0, 1, 2, ... per rank).
   Errors: GVM_EINVAL (type, shape, offsets, non-pinned host buffer),
   GVM_EAGAIN (ring slot or staging space busy: retry after gvm_sync),
   GVM_ENOMEM (can never fit), GVM_ESTATE (detached or shut down),
   GVM_EDEVICE (a CUDA call failed). */
GVM_API int gvm_submit(gvm_rank* rank, const gvm_task* task, uint64_t* seq_out);

/* Submits tasks[0 .. count-1] in order, as count calls of gvm_submit would,
   stopping at the first task that cannot be admitted right now. Returns the
   number submitted (0 .. count) and sets *first_seq to the sequence number of
   tasks[0]; a task that is invalid or can never fit returns its error code
   when it is the first one, else ends the batch early. */
GVM_API int gvm_submit_many(gvm_rank* rank, const gvm_task* tasks, uint32_t count, uint64_t* first_seq);

/* STP() + RCV(): blocks until every task of this rank with sequence <= seq
   is complete and, in host mode, its output is in the host buffer. Results
   become visible to the rank in sequence order (Section 4.2.3 keeps the
   process order). GVM_ETIMEDOUT after wait_timeout_ns without progress,
   GVM_EDEVICE if the scheduler (or, in PS-1/PS-2 mode, the rank's stream)
   reported an error, GVM_EINVAL if seq was never issued, GVM_ESTATE in
   barrier, PS-1 or PS-2 mode if seq was submitted after the last gvm_flush. */
GVM_API int gvm_sync(gvm_rank* rank, uint64_t seq);

/* Non-blocking completion test: 1 if task seq is complete, 0 if not, or a
   negative error code. */
GVM_API int gvm_poll(gvm_rank* rank, uint64_t seq);

/* Barrier mode: launches the scheduler on sched_stream; it drains every task
   submitted (on any rank) before this call and then exits. A task submitted
   after the last flush is not run (gvm_sync on it returns GVM_ESTATE) until
   the next flush. Continuous mode: nothing to do. Returns without waiting.
   Output copies of host-mode tasks are enqueued only after the launch that
   produces them (by gvm_sync / gvm_poll of the owning rank), so a stream wait
   never sits ahead of its producer in a shared hardware queue.
   GVM_MODE_PS1 / GVM_MODE_PS2: enqueues, in the style's order, the copies,
   kernel launches and completion words of every task submitted before this
   call (as in barrier mode, later tasks wait for the next flush). */
GVM_API int gvm_flush(gvm_ctx* ctx);

/* Waits until the scheduler kernel and all copy streams are idle. */
GVM_API int gvm_wait_idle(gvm_ctx* ctx);

/* Copies bytes between host memory and the rank's resident region
   (synchronously, on the rank's input stream). off + bytes must lie inside the
   region. These place the inputs of GVM_TASK_RESIDENT tasks and read their
   outputs back; they are not part of a task. */
GVM_API int gvm_rank_write(gvm_rank* rank, uint64_t off, const void* src, uint64_t bytes);
GVM_API int gvm_rank_read(gvm_rank* rank, uint64_t off, void* dst, uint64_t bytes);

/* The manager's streams (cudaStream_t as void*): which = -1 is the scheduler
   stream, 2r / 2r+1 the input / output stream of rank r. NULL when out of
   range. Valid until gvm_shutdown. */
GVM_API void* gvm_stream(gvm_ctx* ctx, int32_t which);

/* Device address of the rank's resident region (for callers that fill it
   with their own kernels or copies), or NULL for a bad handle. */
GVM_API void* gvm_rank_resident_ptr(gvm_rank* rank);

/* RLS(): waits for the rank's tasks, then releases the rank. Barrier, PS-1
   and PS-2 modes: GVM_ESTATE if some task was submitted after the last
   gvm_flush. */
GVM_API int gvm_detach(gvm_rank* rank);

/* Stops the scheduler after in-flight work, waits for the streams, frees the
   rings and the handle. Tasks never taken from a ring report GVM_ECANCELED
   through gvm_sync from then on (the handle is gone, so callers must not sync
   after shutdown). GVM_ESTATE, with nothing stopped or freed, while a
   gvm_ipc server serves this manager: gvm_ipc_stop it first. */
GVM_API int gvm_shutdown(gvm_ctx* ctx);

/* Copies the manager's counters (gvm_stats above) into *out (caller-owned).
   GVM_EINVAL for a NULL argument; callable at any time before gvm_shutdown. */
GVM_API int gvm_stats_get(gvm_ctx* ctx, gvm_stats* out);

/* Device timestamps (globaltimer, ns) of task seq of this rank: when the
   scheduler took it from the ring and when its last tile finished. Valid
   once the task is complete and until its ring slot is reused. */
GVM_API int gvm_task_times(gvm_rank* rank, uint64_t seq, uint64_t* t_ingest_ns, uint64_t* t_done_ns);

/* ---- SPMD harness --------------------------------------------------------
   Runs `steps` steps of the paper's SPMD pattern (Section 6: every process
   issues its task, the manager runs them together, every process collects its
   result) with one native thread per rank, so that a benchmark measures the
   manager rather than an interpreter's threads. ranks[r] must be attached;
   tasks[r][0 .. counts[r]-1] is rank r's batch, submitted in order every step
   (counts[r] <= ring_depth). A step: all threads submit their batches
   (gvm_submit_many, waiting out GVM_EAGAIN), meet, thread 0 calls gvm_flush
   (barrier mode), each thread syncs its last task, all meet again. In barrier
   mode a batch must fit the rank's ring and staging space at once. Timing
   (each array may be NULL): step_ms_device[i] is CUDA-event time on the
   scheduler stream from before the first submit of step i to after its last
   sync; launch_ms_device[i] the same around step i's gvm_flush (its
   scheduler launch; 0 in continuous mode); step_ms_host[i] the step on the
   host clock. latency_ns (may be NULL, as may any latency_ns[r]) asks for
   each task's latency as the rank sees it: rank r then collects its batch
   task by task in submission order (gvm_sync on each), and
   latency_ns[r][i * counts[r] + j] (steps * counts[r] doubles) is the host
   time from the rank's gvm_submit_many call of step i to the moment
   gvm_sync showed task j of that batch complete (ns, CLOCK_MONOTONIC).
   Returns GVM_OK or the first error any rank saw (the remaining steps are
   skipped). The batch submit call counts as each of its tasks' submit. */
GVM_API int gvm_spmd_run(gvm_ctx* ctx, gvm_rank* const* ranks, const gvm_task* const* tasks,
                         const uint32_t* counts, int32_t nranks, int32_t steps, float* step_ms_device,
                         float* launch_ms_device, double* step_ms_host, double* const* latency_ns);

/* The same pattern with two steps in flight per rank: a rank submits step i
   + 1 (and, in barrier mode, thread 0 flushes it) before it collects the
   results of step i, so the copies of consecutive steps overlap on the host
   link (inputs of one step while the outputs of the one before come back).
   Even steps use tasks_even[r], odd steps tasks_odd[r] (NULL: tasks_even);
   give the two distinct output buffers so that a step's results are not
   overwritten before it is collected. A rank's ring and staging space must
   hold two batches. *total_ms_host = host time from the first submit to the
   last step's results; done_ms_host[i] (may be NULL) = when step i's results
   were all collected, from the same start. Returns GVM_OK or the first error
   any rank saw. */
GVM_API int gvm_spmd_run_overlapped(gvm_ctx* ctx, gvm_rank* const* ranks, const gvm_task* const* tasks_even,
                                    const gvm_task* const* tasks_odd, const uint32_t* counts, int32_t nranks,
                                    int32_t steps, double* total_ms_host, double* done_ms_host);

/* The same with nphases steps in flight per rank (nphases >= 1; 2 is
   gvm_spmd_run_overlapped, 1 collects each step before the next): step i
   uses phases[i % nphases][r], and a rank collects step i after it has
   submitted step i + nphases - 1, so up to nphases steps' copies and
   launches are queued at once. Give each phase its own output buffers. A
   rank's ring and staging space must hold nphases batches. Timings and
   errors as gvm_spmd_run_overlapped; GVM_EINVAL for nphases < 1 or a NULL
   phase. */
GVM_API int gvm_spmd_run_pipelined(gvm_ctx* ctx, gvm_rank* const* ranks, const gvm_task* const* const* phases,
                                   int32_t nphases, const uint32_t* counts, int32_t nranks, int32_t steps,
                                   double* total_ms_host, double* done_ms_host);

/* Open-loop serving harness (continuous mode): one native thread per rank
   submits tasks[r][i] at its scheduled arrival arrival_ns[r][i] (nanoseconds
   after a common start, non-decreasing per rank), keeping at most
   max_inflight of its tasks outstanding (0: as many as the ring admits), and
   reaps completions in order as it goes (gvm_poll between arrivals;
   gvm_sync when it must wait). latency_ns[r][i] (may be NULL) = the moment
   rank r saw task i complete minus its scheduled arrival, so a rank that falls
   behind does not hide queueing delay. *span_ns = from the start to the last
   completion seen. Returns GVM_OK or the first error any rank saw. */
GVM_API int gvm_open_loop_run(gvm_ctx* ctx, gvm_rank* const* ranks, const gvm_task* const* tasks,
                              const uint64_t* const* arrival_ns, const uint32_t* counts, int32_t nranks,
                              uint32_t max_inflight, double* const* latency_ns, double* span_ns);

/* A static, NUL-terminated description of a GVM_* return code ("unknown
   error" for other values); never NULL, needs no handle. */
GVM_API const char* gvm_strerror(int code);

/* ---- the task kernels alone -------------------------------------------- */
/* These run one task's kernel on caller-given device buffers, on the given
   stream, without the manager: the kernels of Table 2 as the manager runs
   them, used for unit parity checks, per-kernel measurement and the plain
   one-context-per-process form of Section 4.1. */

/* c = a + b, n binary32 elements (Table 2, VecAdd). Device pointers; any
   alignment; n >= 0. Returns GVM_EINVAL for n < 0 or NULL with n > 0. */
GVM_API int gvm_vadd_f32(const float* a, const float* b, float* c, int64_t n, void* stream);

/* VMUL alone: c[i] = a[i] * b[i]^iters (iters binary32 products, each rounded
   to nearest), n elements, device pointers, on stream (cudaStream_t or NULL).
   GVM_EINVAL for n < 0, iters outside 1 .. 1024 or NULL pointers. */
GVM_API int gvm_vmul_f32(const float* a, const float* b, float* c, int64_t n, int32_t iters, void* stream);

/* Scratch bytes gvm_sgemm_f32 needs for (m, n, k, path): 0 for the FMA path;
   for split3 the bf16 hi/lo copies of A (m x kp) and of B transposed
   (n x kp), kp = k rounded up to a multiple of 8. */
GVM_API uint64_t gvm_sgemm_scratch_bytes(int32_t m, int32_t n, int32_t k, int32_t path);

/* C = A B (Table 2, MM), row-major binary32 device buffers A (m x k), B (k x n),
   C (m x n). path selects the arithmetic; scratch (device, 256-byte aligned,
   >= gvm_sgemm_scratch_bytes) is needed by the split3 path only. Returns
   GVM_EINVAL for bad shapes or a short scratch buffer. */
GVM_API int gvm_sgemm_f32(const float* A, const float* B, float* C, int32_t m, int32_t n, int32_t k,
                  int32_t path, void* scratch, uint64_t scratch_bytes, void* stream);

/* C = A B on the split3 path without any scratch from the caller. The paper
   has no counterpart: this entry point exists for callers that cannot
   allocate device memory -- a plain C program with no device allocator of its
   own, a framework whose pool already owns all device memory, a
   latency-critical loop where allocating is not allowed. It never calls
   cudaMalloc, cudaFree or any allocating routine.

   Scratch: a fixed 32 MiB array in the library's device image, held by every
   GPU that loads the library until the process exits. That bounds the shape:
   4 * (m + n) * kp bytes (kp = k rounded up to 8) must fit, e.g. up to
   m = n = k = 2048; larger shapes return GVM_ENOMEM and launch nothing.
   The first call on a device looks up the array's device address
   (cudaGetSymbolAddress, with that device current) and caches it with the
   id of the device's context; make that first call before any stream
   capture. A call in a new context of the device (after cudaDeviceReset)
   repeats the lookup, so make it before any capture too.

   Every call shares the one array, and the array keeps the previous call's
   contents (each call rewrites every byte it reads, so nothing needs
   clearing). Calls whose kernels overlap on the GPU -- for example on two
   streams at once -- race on the array: order them on one stream.
   Arguments, layout and errors are otherwise those of gvm_sgemm_f32. */
GVM_API int gvm_sgemm_f32_noalloc(const float* A, const float* B, float* C, int32_t m, int32_t n, int32_t k,
                                  void* stream);

/* Reads and clears the error status of the standalone kernels: 0 when every
   bounded wait since the last call finished in time; otherwise the low byte
   is the status and the next byte names the wait. Synchronous. */
GVM_API int gvm_kernel_status(uint32_t* out);

#ifdef __cplusplus
}
#endif
#endif /* GVM_H */
