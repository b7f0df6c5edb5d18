/*
 * gvm_ipc.h -- cross-process ranks for the GPU virtualization manager.
 *
 * The paper's SPMD processes are separate programs: each reaches the GPU
 * virtualization manager (GVM, Section 5) through request and response
 * queues, and its data through a region the GVM shares with it. Here every
 * rank owns one POSIX shared-memory segment, named "/<name>.<rank>":
 *
 *   header   request ring (client -> manager), the rank's counters
 *   data     the rank's operands and results; the manager page-locks it
 *            (cudaHostRegister) so that copies move straight between this
 *            memory and the GPU
 *
 * A client maps only its own segment, so no rank can read or write another
 * rank's buffers (the operating system enforces it). The manager process
 * owns the CUDA context and the gvm_ctx; one serving thread takes each
 * rank's requests (gvm_submit_many with host pointers into the rank's data
 * area), publishes completions, and in barrier, PS-1 and PS-2 modes runs the
 * request barrier across processes: gvm_flush once every attached client has
 * arrived. Client calls make no CUDA call and need no GPU.
 *
 * Lifetime: gvm_ipc_create (segments) -> gvm_ipc_serve (register, attach
 * ranks, start the thread) -> clients open/submit/barrier/wait/close ->
 * gvm_ipc_stop -> gvm_ipc_destroy (unlink). Errors are the GVM_* codes of
 * gvm.h.
 */
#ifndef GVM_IPC_H
#define GVM_IPC_H

#include "gvm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gvm_ipc_region gvm_ipc_region; /* manager side: the segments */
typedef struct gvm_ipc_server gvm_ipc_server; /* manager side: the serving thread */
typedef struct gvm_ipc_client gvm_ipc_client; /* client side: one rank's mapping */

/* One request. Operands and result are given as byte offsets into the rank's
   data area; each must lie inside it (checked by the manager, which refuses
   the task with GVM_EINVAL otherwise). Alignment and sizes as gvm_task: 4
   bytes for vector tasks, 16 for SGEMM. */
typedef struct gvm_ipc_task {
  int32_t type;     /* GVM_TASK_VADD, GVM_TASK_VMUL or GVM_TASK_SGEMM */
  int32_t reserved; /* 0 */
  int64_t m, n, k;  /* as gvm_task (VMUL: k = products per element) */
  uint64_t a_off, b_off, c_off;
} gvm_ipc_task;

/* Rank state in the segment header. */
#define GVM_IPC_FREE 0     /* no client */
#define GVM_IPC_ATTACHED 1 /* a client has it open */
#define GVM_IPC_CLOSED 2   /* the client closed it */
#define GVM_IPC_LOST 3     /* the client process ended without closing */

/* Creates nranks segments "/<name>.<rank>" (name: 1..40 characters of
   [A-Za-z0-9_-]), each with a request ring of `depth` entries (power of two,
   2..4096) and a data area of data_bytes (rounded up to 2 MiB), reserved in
   full now (GVM_ENOMEM if the shared-memory file system cannot hold it).
   Fails with GVM_EBUSY if a segment of that name exists. */
GVM_API int gvm_ipc_create(const char* name, int32_t nranks, uint64_t data_bytes, int32_t depth,
                           gvm_ipc_region** out);

/* Unlocks (if it was served) the data areas, unmaps and unlinks the
   segments. The region must not be served; call it after gvm_shutdown of the
   manager that served it (a continuous-mode scheduler holds the device until
   then, and unlocking host memory may wait for the device). */
GVM_API int gvm_ipc_destroy(gvm_ipc_region* region);

/* Serves the region with manager ctx (created with max_ranks >= nranks; ranks
   0..nranks-1 must not be attached): page-locks every data area, attaches
   the ranks and starts the serving thread. A rank's request numbers are the
   manager rank's sequence numbers, so the region must be fresh. */
GVM_API int gvm_ipc_serve(gvm_ctx* ctx, gvm_ipc_region* region, gvm_ipc_server** out);

/* Stops taking requests, runs a last request barrier for what was taken,
   waits for every taken task (bounded by the manager's wait_timeout_ns) and
   detaches the ranks; the data areas stay page-locked until gvm_ipc_destroy.
   Requests not yet taken are dropped; their clients see GVM_ECANCELED. A
   region is served once (GVM_ESTATE for a second gvm_ipc_serve). */
GVM_API int gvm_ipc_stop(gvm_ipc_server* server);

/* Requests taken and completed over all ranks, barriers run. */
GVM_API int gvm_ipc_server_counts(gvm_ipc_server* server, uint64_t* taken, uint64_t* completed,
                                  uint64_t* barriers);

/* Diagnostic read of rank `rank`'s header counters (no lock). */
GVM_API int gvm_ipc_peek(gvm_ipc_region* region, int32_t rank, uint64_t* head, uint64_t* arrived,
                         uint64_t* done, uint32_t* state);

/* ---- client side (any process; no CUDA call) ---------------------------- */

/* Maps segment "/<name>.<rank>" and marks it attached by this process.
   GVM_EINVAL: no such segment or not a gvm segment; GVM_EBUSY: another live
   process has it open. */
GVM_API int gvm_ipc_open(const char* name, int32_t rank, gvm_ipc_client** out);

/* The rank's data area (page-aligned) and its size; NULL for a bad handle. */
GVM_API void* gvm_ipc_data(gvm_ipc_client* client, uint64_t* bytes);

/* Appends one request; *seq = its sequence number (0, 1, ... per rank, over
   the segment's life). GVM_EAGAIN when the ring is full (wait on an earlier
   task first). The operand bytes must be in the data area before the call
   and stay untouched until gvm_ipc_wait returns for the task. */
GVM_API int gvm_ipc_submit(gvm_ipc_client* client, const gvm_ipc_task* task, uint64_t* seq);

/* Arrives at the request barrier: every request submitted before this call
   runs at the next barrier the manager runs (in continuous mode requests run
   without one, and this call only records the arrival). */
GVM_API int gvm_ipc_barrier(gvm_ipc_client* client);

/* Blocks until task seq is complete and its result is in the data area.
   GVM_ETIMEDOUT after timeout_ns (0: no limit), the manager's error code if
   it refused or failed the task, GVM_ECANCELED if the manager stopped or its
   process ended. */
GVM_API int gvm_ipc_wait(gvm_ipc_client* client, uint64_t seq, uint64_t timeout_ns);

/* Marks the rank closed and unmaps it (outstanding tasks still run). */
GVM_API int gvm_ipc_close(gvm_ipc_client* client);

#ifdef __cplusplus
}
#endif

#endif /* GVM_IPC_H */
