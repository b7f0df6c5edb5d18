// Host runtime of the GPU virtualization manager: the C ABI of gvm.h.
//
// One manager owns one device context (the caller's) and serves many ranks,
// the paper's single daemon with one virtual GPU per SPMD process (Section 5).
// Per rank it keeps:
//   - a ring of task descriptors in pinned host memory, read by the
//     scheduler kernel (the paper's request queue);
//   - a slice of the caller's device arena: a resident region addressed by
//     task offsets and a staging ring for copied operands (the
//     paper's per-process memory objects, so ranks never share buffers);
//   - an input stream and an output stream (the paper's one stream per
//     process): input copies then a ready word; a wait on the task's done
//     word then the output copy and the completion word.
// Resident-mode tasks use no stream at all: the scheduler reads the ring and
// writes the completion word itself.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/prctl.h>

#include <atomic>
#include <chrono>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "gvm.h"
#include "gvm_internal.h"
#include "gvm_runtime.h"

using namespace gvm;

namespace {

struct SlotInfo {
  uint64_t stage_end = 0;  // staging-ring counter after this task's allocation
  uint64_t bytes = 0;      // staging bytes this task holds (incl. wrap waste)
  // Output operations of a host-mode task, pushed on the rank's output stream
  // only after the scheduler launch that will write its done word.
  void* c_host = nullptr;
  uint64_t c_dev = 0;
  uint64_t c_bytes = 0;
  bool needs_out = false;
  // PS-1 / PS-2 modes: the task's own input copies, issued by gvm_flush.
  const void* a_host = nullptr;
  const void* b_host = nullptr;
  uint64_t a_dev = 0, b_dev = 0, a_bytes = 0, b_bytes = 0;
  bool host_io = false;
  // Output in pageable host memory: the task completes on the device with
  // its result in staging; reap copies it out before reporting it.
  bool out_pageable = false;
};

inline uint32_t tag_of(uint64_t seq) { return (uint32_t)(seq + 1); }

// GVM_DEBUG=1 in the environment traces manager state changes on stderr.
bool debug_on() {
  static const bool on = getenv("GVM_DEBUG") != nullptr;
  return on;
}
#define GVM_TRACE(...)                     \
  do {                                     \
    if (debug_on()) {                      \
      fprintf(stderr, "[gvm] " __VA_ARGS__); \
      fputc('\n', stderr);                 \
    }                                      \
  } while (0)

// gvm_sync gives the device this long beyond its own wait limit to report.
constexpr uint64_t kStreamQueryNs = 2000000;  // gvm_sync: driver status check period (2 ms)
constexpr uint64_t kSyncSpinNs = 5000000;     // gvm_sync: spin this long, then sleep between polls
constexpr uint64_t kSyncSleepNs = 10000;      // gvm_sync: poll period once sleeping
// Copies of one batch are merged when both sides are adjacent, by default up
// to this many bytes per copy (gvm_config.copy_run_bytes): the link serves
// 1 MiB copies at less than half its rate, while a few MiB per copy still
// lets the scheduler start on the first tasks while later inputs arrive.
constexpr uint64_t kDefaultCopyRun = 16ull << 20;
constexpr uint64_t kHostGraceNs = 1000ull * 1000 * 1000;

// Sleeps about ns nanoseconds: the calling thread's timer slack is set to
// 1 us the first time (the default 50 us would stretch every short sleep).
inline void short_sleep(uint64_t ns) {
  thread_local bool slack_set = false;
  if (!slack_set) {
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
    slack_set = true;
  }
  std::this_thread::sleep_for(std::chrono::nanoseconds(ns));
}

inline uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

struct gvm_rank {
  gvm_ctx* ctx = nullptr;
  int32_t id = 0;
  bool attached = false;
  uint64_t next_seq = 0;  // sequence number of the next submission
  uint64_t synced = 0;    // tasks 0 .. synced-1 are known complete
  uint64_t out_pushed = 0;           // tasks whose output operations are on the output stream
  std::atomic<uint64_t> published{0};  // next_seq as seen by gvm_flush
  std::atomic<uint64_t> flushed{0};    // barrier mode: tasks covered by a launched flush
  uint64_t slice = 0;     // device address of the rank's slice
  uint64_t ring_base = 0, ring_bytes = 0;
  uint64_t ring_head = 0, ring_tail = 0;  // monotonic byte counters
  std::vector<SlotInfo> slots;
  bool copy_failed = false;  // a pageable output could not be copied out
  cudaStream_t in_stream = nullptr, out_stream = nullptr;
  std::mutex mu;
};

struct gvm_ctx {
  gvm_config cfg{};
  CtrlLayout L{};
  int path = kPathFma;
  int grid = 0;
  size_t smem = 0;
  uint64_t slice_bytes = 0;
  uint8_t* host_block = nullptr;
  HostHead* heads = nullptr;
  TaskBody* descs = nullptr;
  HostComplete* completes = nullptr;
  HostShared* shared = nullptr;
  SchedParams params{};
  cudaStream_t sched = nullptr;
  std::vector<std::unique_ptr<gvm_rank>> ranks;
  std::mutex launch_mu;
  uint32_t launch_gen = 0;
  std::atomic<uint64_t> staged{0}, staged_peak{0}, submitted{0}, completed{0}, h2d{0}, d2h{0}, launches{0};
  bool shut = false;
  std::atomic<int> ipc_servers{0};  // gvm_ipc servers using this manager
  int device = 0;
  std::vector<cudaStream_t> owned_streams;  // created by gvm_init, destroyed by gvm_shutdown
  ~gvm_ctx() {
    for (cudaStream_t st : owned_streams) cudaStreamDestroy(st);
  }
};

namespace gvm {
int ctx_mode(const gvm_ctx* ctx) { return ctx->cfg.mode; }
int ctx_max_ranks(const gvm_ctx* ctx) { return ctx->cfg.max_ranks; }
void ctx_servers_add(gvm_ctx* ctx, int delta) { ctx->ipc_servers.fetch_add(delta, std::memory_order_acq_rel); }
}  // namespace gvm

namespace {

bool cfg_valid(const gvm_config* c) {
  if (!c) return false;
  if (c->max_ranks < 1 || c->max_ranks > GVM_MAX_RANKS) return false;
  if (c->ring_depth < 2 || c->ring_depth > 4096 || (c->ring_depth & (c->ring_depth - 1))) return false;
  if (c->mode != GVM_MODE_BARRIER && c->mode != GVM_MODE_CONTINUOUS && c->mode != GVM_MODE_PS1 &&
      c->mode != GVM_MODE_PS2)
    return false;
  if (c->sgemm_path != GVM_SGEMM_FMA && c->sgemm_path != GVM_SGEMM_SPLIT3 && c->sgemm_path != GVM_SGEMM_SPLIT3_WIDE &&
      c->sgemm_path != GVM_SGEMM_SPLIT3_TMA)
    return false;
  return true;
}

// PS-1 / PS-2: the host issues each task's copies and kernel (no scheduler).
inline bool stream_mode(const gvm_ctx* ctx) {
  return ctx->cfg.mode == GVM_MODE_PS1 || ctx->cfg.mode == GVM_MODE_PS2;
}

// Modes in which a task runs only after a gvm_flush that follows it.
inline bool flush_mode(const gvm_ctx* ctx) { return ctx->cfg.mode != GVM_MODE_CONTINUOUS; }

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return GVM_OK;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return GVM_ENODEV;
  return GVM_EDEVICE;
}

uint32_t ld_acq(const uint32_t* p) { return __atomic_load_n(p, __ATOMIC_ACQUIRE); }

// Makes the manager's device (its primary context) current in the calling
// thread before CUDA or driver calls: rank threads may never have touched
// CUDA themselves.
thread_local bool tl_bound = false;
inline void bind_device(const gvm_ctx* ctx) {
  int d = -1;
  if (!tl_bound || cudaGetDevice(&d) != cudaSuccess || d != ctx->device) {
    cudaSetDevice(ctx->device);
    tl_bound = true;
  }
}

// Launch the scheduler once (caller holds launch_mu).
int launch_locked(gvm_ctx* ctx, uint32_t drain) {
  ctx->launch_gen += 1;
  SchedParams p = ctx->params;
  p.drain = drain;
  p.launch_gen = ctx->launch_gen;
  cudaError_t e = launch_scheduler(ctx->path, p, ctx->grid, ctx->smem, ctx->sched);
  if (e != cudaSuccess) return GVM_EDEVICE;
  ctx->launches.fetch_add(1);
  return GVM_OK;
}

// Advance `synced` over completed tasks and release their staging bytes.
void reap(gvm_rank* r) {
  gvm_ctx* ctx = r->ctx;
  const uint32_t D = (uint32_t)ctx->cfg.ring_depth;
  while (r->synced < r->next_seq) {
    const uint64_t s = r->synced;
    const uint32_t idx = (uint32_t)r->id * D + (uint32_t)(s & (D - 1));
    if (ld_acq(&ctx->completes[idx].tag) != tag_of(s)) break;
    SlotInfo& si = r->slots[s & (D - 1)];
    if (si.out_pageable) {
      // The result waits in staging: copy it to the caller's pageable buffer
      // now (the input stream carries only copies, so waiting on it ends).
      cudaError_t e = cudaMemcpyAsync(si.c_host, reinterpret_cast<const void*>(si.c_dev), si.c_bytes,
                                      cudaMemcpyDeviceToHost, r->in_stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(r->in_stream);
      if (e != cudaSuccess) {
        r->copy_failed = true;
        break;
      }
      ctx->d2h.fetch_add(si.c_bytes);
      si.out_pageable = false;
    }
    if (si.bytes) {
      r->ring_tail = si.stage_end;
      ctx->staged.fetch_sub(si.bytes);
      si.bytes = 0;
    }
    r->synced = s + 1;
    ctx->completed.fetch_add(1);
  }
}

// A copy between a host buffer (src) and staging (dst) still to issue, or a
// run of adjacent ones.
struct CopyRun {
  uint64_t dst;
  const uint8_t* src;
  uint64_t bytes;
  uint32_t first_piece, pieces;  // the operand copies it merges
};

// Issues one merged copy. Host buffers that are adjacent may still be
// separate page-locked allocations, which one copy may not span (the call
// fails with cudaErrorInvalidValue and enqueues nothing): then the run's
// operand copies are issued one by one.
cudaError_t issue_run(const CopyRun& run, const std::vector<CopyRun>& pieces, cudaMemcpyKind kind,
                      cudaStream_t st) {
  void* dst = kind == cudaMemcpyHostToDevice ? reinterpret_cast<void*>(run.dst) : const_cast<uint8_t*>(run.src);
  const void* src = kind == cudaMemcpyHostToDevice ? static_cast<const void*>(run.src)
                                                   : reinterpret_cast<const void*>(run.dst);
  cudaError_t e = cudaMemcpyAsync(dst, src, run.bytes, kind, st);
  if (e != cudaErrorInvalidValue || run.pieces < 2) return e;
  (void)cudaGetLastError();
  for (uint32_t i = 0; i < run.pieces; ++i) {
    const CopyRun& p = pieces[run.first_piece + i];
    void* d = kind == cudaMemcpyHostToDevice ? reinterpret_cast<void*>(p.dst) : const_cast<uint8_t*>(p.src);
    const void* s = kind == cudaMemcpyHostToDevice ? static_cast<const void*>(p.src)
                                                   : reinterpret_cast<const void*>(p.dst);
    e = cudaMemcpyAsync(d, s, p.bytes, kind, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Pushes the output operations of tasks out_pushed .. upto-1 on the rank's
// output stream: a wait on each task's done word, the device-to-host copy of
// its output, its completion word. Outputs adjacent on both sides (a batch's
// outputs are packed in staging; adjacent host buffers are the caller's
// choice) share one copy of up to copy_run_bytes after all their waits.
// Called only once the scheduler launch that will write those done words has
// been pushed: a blocked wait can then never sit ahead of its own producer in
// a hardware queue that two streams share.
int push_out_ops(gvm_rank* r, uint64_t upto) {
  gvm_ctx* ctx = r->ctx;
  const DriverApi* api = driver_api();
  const uint32_t D = (uint32_t)ctx->cfg.ring_depth;
  CUstream os = reinterpret_cast<CUstream>(r->out_stream);
  while (r->out_pushed < upto) {
    const uint64_t s0 = r->out_pushed;
    SlotInfo& first = r->slots[s0 & (D - 1)];
    if (!first.needs_out) {
      r->out_pushed = s0 + 1;
      continue;
    }
    // The run: s0 .. s1-1, outputs adjacent in device and host memory.
    std::vector<CopyRun> pieces;
    pieces.push_back(CopyRun{first.c_dev, static_cast<const uint8_t*>(first.c_host), first.c_bytes, 0, 1});
    uint64_t s1 = s0 + 1, bytes = first.c_bytes;
    while (s1 < upto) {
      const SlotInfo& nx = r->slots[s1 & (D - 1)];
      if (!nx.needs_out || nx.c_dev != first.c_dev + bytes ||
          static_cast<const uint8_t*>(nx.c_host) != static_cast<const uint8_t*>(first.c_host) + bytes ||
          bytes + nx.c_bytes > ctx->cfg.copy_run_bytes)
        break;
      pieces.push_back(CopyRun{nx.c_dev, static_cast<const uint8_t*>(nx.c_host), nx.c_bytes, 0, 1});
      bytes += nx.c_bytes;
      ++s1;
    }
    const CopyRun run{first.c_dev, static_cast<const uint8_t*>(first.c_host), bytes, 0, (uint32_t)pieces.size()};
    for (uint64_t s = s0; s < s1; ++s) {
      const uint32_t idx = (uint32_t)r->id * D + (uint32_t)(s & (D - 1));
      if (api->wait_value32(os, reinterpret_cast<CUdeviceptr>(ctx->params.done + idx), tag_of(s),
                            CU_STREAM_WAIT_VALUE_EQ) != CUDA_SUCCESS)
        return GVM_EDEVICE;
    }
    if (bytes && issue_run(run, pieces, cudaMemcpyDeviceToHost, r->out_stream) != cudaSuccess) return GVM_EDEVICE;
    for (uint64_t s = s0; s < s1; ++s) {
      const uint32_t idx = (uint32_t)r->id * D + (uint32_t)(s & (D - 1));
      if (api->write_value32(os, reinterpret_cast<CUdeviceptr>(&ctx->params.host_complete[idx].tag), tag_of(s),
                             CU_STREAM_WRITE_VALUE_DEFAULT) != CUDA_SUCCESS)
        return GVM_EDEVICE;
      r->slots[s & (D - 1)].needs_out = false;
    }
    ctx->d2h.fetch_add(bytes);
    r->out_pushed = s1;
  }
  return GVM_OK;
}

// Barrier mode: output operations for the tasks covered by a launched flush.
int push_flushed(gvm_rank* r) {
  if (r->ctx->cfg.mode != GVM_MODE_BARRIER) return GVM_OK;
  const uint64_t f = std::min(r->flushed.load(std::memory_order_acquire), r->next_seq);
  return push_out_ops(r, f);
}

// Bounded wait for the scheduler stream (wait_timeout_ns plus a grace
// period). On timeout the device control block is read back on a separate
// stream and traced, and GVM_ETIMEDOUT is returned.
int wait_scheduler(gvm_ctx* ctx) {
  const uint64_t t0 = now_ns();
  while (true) {
    const cudaError_t e = cudaStreamQuery(ctx->sched);
    if (e == cudaSuccess) return GVM_OK;
    if (e != cudaErrorNotReady) return GVM_EDEVICE;
    if (now_ns() - t0 > ctx->cfg.wait_timeout_ns + kHostGraceNs) break;
    std::this_thread::yield();
  }
  DevCtrl c;
  memset(&c, 0, sizeof(c));
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess) {
    if (cudaMemcpyAsync(&c, ctx->params.ctrl, sizeof(c), cudaMemcpyDeviceToHost, s) == cudaSuccess)
      cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  fprintf(stderr,
          "[gvm] scheduler did not stop: lock=%u abort=%u exit_count=%u drained=%u published=%llu "
          "tiles=%llu next_tile=%llu consumed=%llu status=%u\n",
          c.ingest_lock, c.abort, c.exit_count, c.drained, (unsigned long long)c.published,
          (unsigned long long)c.published_tiles, (unsigned long long)c.next_tile, (unsigned long long)c.cursor,
          ld_acq(&ctx->shared->status));
  return GVM_ETIMEDOUT;
}

// ---- PS-1 / PS-2 (Section 4.2.1): the host issues every task's own work.

// Input copies of task s, one per operand, on the rank's stream.
int ps_issue_in(gvm_rank* r, uint64_t s) {
  gvm_ctx* ctx = r->ctx;
  const SlotInfo& si = r->slots[s & (uint64_t)(ctx->cfg.ring_depth - 1)];
  if (!si.host_io) return GVM_OK;
  if (si.a_bytes && cudaMemcpyAsync(reinterpret_cast<void*>(si.a_dev), si.a_host, si.a_bytes,
                                    cudaMemcpyHostToDevice, r->in_stream) != cudaSuccess)
    return GVM_EDEVICE;
  if (si.b_bytes && cudaMemcpyAsync(reinterpret_cast<void*>(si.b_dev), si.b_host, si.b_bytes,
                                    cudaMemcpyHostToDevice, r->in_stream) != cudaSuccess)
    return GVM_EDEVICE;
  ctx->h2d.fetch_add(si.a_bytes + si.b_bytes);
  return GVM_OK;
}

// The task's kernel, launched alone on the rank's stream.
int ps_issue_comp(gvm_rank* r, uint64_t s) {
  gvm_ctx* ctx = r->ctx;
  const uint32_t D = (uint32_t)ctx->cfg.ring_depth;
  const TaskBody& b = ctx->descs[(uint32_t)r->id * D + (uint32_t)(s & (D - 1))];
  const float* A = reinterpret_cast<const float*>(b.a);
  const float* B = reinterpret_cast<const float*>(b.b);
  float* C = reinterpret_cast<float*>(b.c);
  int rc = GVM_OK;
  if (b.type == kTaskVadd) {
    if (b.n == 0) return GVM_OK;
    rc = gvm_vadd_f32(A, B, C, b.n, r->in_stream);
  } else if (b.type == kTaskVmul) {
    if (b.n == 0) return GVM_OK;
    rc = gvm_vmul_f32(A, B, C, b.n, b.k, r->in_stream);
  } else {
    // The fused split3 form needs no scratch and computes the same tiles as
    // the scheduler's split3 path.
    const int path = (ctx->path == kPathSplit3 || ctx->path == kPathSplit3Tma) ? GVM_SGEMM_SPLIT3_FUSED
                     : ctx->path == kPathSplit3Wide                             ? GVM_SGEMM_SPLIT3_WIDE
                                                                                : GVM_SGEMM_FMA;
    rc = gvm_sgemm_f32(A, B, C, b.m, (int32_t)b.n, b.k, path, nullptr, 0, r->in_stream);
  }
  if (rc == GVM_OK) ctx->launches.fetch_add(1);
  return rc;
}

// Output copy of task s, then its completion word.
int ps_issue_out(gvm_rank* r, uint64_t s) {
  gvm_ctx* ctx = r->ctx;
  const uint32_t D = (uint32_t)ctx->cfg.ring_depth;
  const SlotInfo& si = r->slots[s & (D - 1)];
  if (si.host_io && si.c_bytes) {
    if (cudaMemcpyAsync(si.c_host, reinterpret_cast<const void*>(si.c_dev), si.c_bytes, cudaMemcpyDeviceToHost,
                        r->in_stream) != cudaSuccess)
      return GVM_EDEVICE;
    ctx->d2h.fetch_add(si.c_bytes);
  }
  const uint32_t idx = (uint32_t)r->id * D + (uint32_t)(s & (D - 1));
  if (driver_api()->write_value32(reinterpret_cast<CUstream>(r->in_stream),
                                  reinterpret_cast<CUdeviceptr>(&ctx->params.host_complete[idx].tag), tag_of(s),
                                  CU_STREAM_WRITE_VALUE_DEFAULT) != CUDA_SUCCESS)
    return GVM_EDEVICE;
  return GVM_OK;
}

// The request barrier of PS-1 / PS-2: every task published before this call
// and not yet issued, in the style's order. PS-1: all ranks' input copies,
// then all kernels, then all output copies (within a rank, task order). PS-2:
// rank by rank, task by task, input -> kernel -> output. Each rank's work goes
// on its own stream, so the hardware overlaps what the style allows. Caller
// holds launch_mu.
int ps_flush_locked(gvm_ctx* ctx) {
  const size_t R = ctx->ranks.size();
  std::vector<uint64_t> from(R), upto(R);
  for (size_t i = 0; i < R; ++i) {
    upto[i] = ctx->ranks[i]->published.load(std::memory_order_acquire);
    from[i] = std::min(ctx->ranks[i]->flushed.load(std::memory_order_acquire), upto[i]);
  }
  int rc = GVM_OK;
  if (ctx->cfg.mode == GVM_MODE_PS1) {
    for (int phase = 0; phase < 3 && rc == GVM_OK; ++phase)
      for (size_t i = 0; i < R && rc == GVM_OK; ++i)
        for (uint64_t s = from[i]; s < upto[i] && rc == GVM_OK; ++s) {
          gvm_rank* r = ctx->ranks[i].get();
          rc = phase == 0 ? ps_issue_in(r, s) : phase == 1 ? ps_issue_comp(r, s) : ps_issue_out(r, s);
        }
  } else {
    for (size_t i = 0; i < R && rc == GVM_OK; ++i)
      for (uint64_t s = from[i]; s < upto[i] && rc == GVM_OK; ++s) {
        gvm_rank* r = ctx->ranks[i].get();
        rc = ps_issue_in(r, s);
        if (rc == GVM_OK) rc = ps_issue_comp(r, s);
        if (rc == GVM_OK) rc = ps_issue_out(r, s);
      }
  }
  if (rc != GVM_OK) return rc;
  for (size_t i = 0; i < R; ++i) ctx->ranks[i]->flushed.store(upto[i], std::memory_order_release);
  return GVM_OK;
}

// 1: page-locked host memory; 0: pageable host memory; -1: device or managed
// memory, which a task may not name (a rank reaches the GPU only through the
// manager's copies).
int host_kind(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  if (a.type == cudaMemoryTypeHost) return 1;
  if (a.type == cudaMemoryTypeUnregistered) return 0;
  return -1;
}

}  // namespace

extern "C" {

uint64_t gvm_ctrl_bytes(const gvm_config* cfg) {
  if (!cfg_valid(cfg)) return 0;
  return ctrl_layout((uint32_t)cfg->max_ranks, (uint32_t)cfg->ring_depth).total;
}

const char* gvm_strerror(int code) {
  switch (code) {
    case GVM_OK: return "ok";
    case GVM_EINVAL: return "invalid argument";
    case GVM_EBUSY: return "rank already attached";
    case GVM_EAGAIN: return "ring slot or staging space busy, retry after gvm_sync";
    case GVM_ENOMEM: return "task can never fit the rank's staging space or the admission cap";
    case GVM_ETIMEDOUT: return "bounded wait ran out";
    case GVM_EDEVICE: return "CUDA call failed or device reported an error";
    case GVM_ECANCELED: return "manager shut down";
    case GVM_ESTATE: return "call not valid in the current state";
    case GVM_ENODEV: return "no usable CUDA device";
    default: return "unknown error";
  }
}

int gvm_init(const gvm_config* cfg_in, gvm_ctx** out) {
  if (!out || !cfg_valid(cfg_in)) return GVM_EINVAL;
  *out = nullptr;
  gvm_config cfg = *cfg_in;
  if (!cfg.arena || (reinterpret_cast<uintptr_t>(cfg.arena) & 255)) return GVM_EINVAL;
  if (!cfg.ctrl || (reinterpret_cast<uintptr_t>(cfg.ctrl) & 255)) return GVM_EINVAL;
  const CtrlLayout L = ctrl_layout((uint32_t)cfg.max_ranks, (uint32_t)cfg.ring_depth);
  if (cfg.ctrl_bytes < L.total) return GVM_EINVAL;
  const uint64_t slice = (cfg.arena_bytes / (uint64_t)cfg.max_ranks) & ~uint64_t(255);
  const uint64_t resident = align_up(cfg.resident_bytes, 256);
  if (slice == 0 || resident > slice) return GVM_EINVAL;
  if (cfg.wait_timeout_ns == 0) cfg.wait_timeout_ns = 10ull * 1000 * 1000 * 1000;
  if (cfg.idle_poll_ns == 0) cfg.idle_poll_ns = 1000;
  if (cfg.copy_run_bytes == 0) cfg.copy_run_bytes = kDefaultCopyRun;
  if (cfg.vadd_tile < 0) return GVM_EINVAL;
  if (cfg.direct_output < 0 || cfg.direct_output > 1 || cfg.l2_prefetch < 0 || cfg.l2_prefetch > 1 ||
      cfg.copy_streams_max < 0 || cfg.copy_in_streams < 0)
    return GVM_EINVAL;
  if (cfg.vadd_tile > 0) cfg.vadd_tile = std::max<int64_t>(1024, cfg.vadd_tile / 1024 * 1024);
  if (cfg.ingest_quantum <= 0) cfg.ingest_quantum = 4;
  if (cfg.copy_streams)
    for (int i = 0; i < 2 * cfg.max_ranks; ++i)
      if (!cfg.copy_streams[i]) return GVM_EINVAL;
  if (!driver_api()) return GVM_ENODEV;

  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e);
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_err(e);

  auto ctx = std::make_unique<gvm_ctx>();
  ctx->cfg = cfg;
  ctx->L = L;
  ctx->path = cfg.sgemm_path == GVM_SGEMM_SPLIT3        ? kPathSplit3
              : cfg.sgemm_path == GVM_SGEMM_SPLIT3_WIDE ? kPathSplit3Wide
              : cfg.sgemm_path == GVM_SGEMM_SPLIT3_TMA  ? kPathSplit3Tma
                                                        : kPathFma;
  ctx->slice_bytes = slice;
  ctx->device = dev;
  if (cfg.sched_stream) {
    ctx->sched = static_cast<cudaStream_t>(cfg.sched_stream);
  } else {
    e = cudaStreamCreateWithFlags(&ctx->sched, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_err(e);
    ctx->owned_streams.push_back(ctx->sched);
  }
  int bps = 0;
  e = scheduler_setup(ctx->path, &bps, &ctx->smem);
  if (e != cudaSuccess) return cuda_err(e);
  if (bps < 1) return GVM_EDEVICE;
  ctx->grid = cfg.grid_ctas > 0 ? std::min(cfg.grid_ctas, sms * bps) : sms * bps;

  const uint32_t R = (uint32_t)cfg.max_ranks, D = (uint32_t)cfg.ring_depth;
  const uint64_t slots = (uint64_t)R * D;
  const uint64_t off_heads = 0;
  const uint64_t off_descs = align_up(off_heads + sizeof(HostHead) * R, 128);
  const uint64_t off_comp = align_up(off_descs + sizeof(TaskBody) * slots, 128);
  const uint64_t off_shared = align_up(off_comp + sizeof(HostComplete) * slots, 128);
  const uint64_t host_total = align_up(off_shared + sizeof(HostShared), 4096);
  void* hb = nullptr;
  e = cudaHostAlloc(&hb, host_total, cudaHostAllocMapped | cudaHostAllocPortable);
  if (e != cudaSuccess) return GVM_ENOMEM;
  memset(hb, 0, host_total);
  ctx->host_block = static_cast<uint8_t*>(hb);
  ctx->heads = reinterpret_cast<HostHead*>(ctx->host_block + off_heads);
  ctx->descs = reinterpret_cast<TaskBody*>(ctx->host_block + off_descs);
  ctx->completes = reinterpret_cast<HostComplete*>(ctx->host_block + off_comp);
  ctx->shared = reinterpret_cast<HostShared*>(ctx->host_block + off_shared);
  void* dhb = nullptr;
  e = cudaHostGetDevicePointer(&dhb, hb, 0);
  if (e != cudaSuccess) {
    cudaFreeHost(hb);
    return GVM_EDEVICE;
  }
  uint8_t* dh = static_cast<uint8_t*>(dhb);

  uint8_t* dc = static_cast<uint8_t*>(cfg.ctrl);
  e = cudaMemsetAsync(dc, 0, L.total, ctx->sched);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->sched);
  if (e != cudaSuccess) {
    cudaFreeHost(hb);
    return GVM_EDEVICE;
  }
  SchedParams& p = ctx->params;
  p.ctrl = reinterpret_cast<DevCtrl*>(dc);
  p.tail = reinterpret_cast<uint32_t*>(dc + L.off_tail);
  p.ready = reinterpret_cast<uint32_t*>(dc + L.off_ready);
  p.done = reinterpret_cast<uint32_t*>(dc + L.off_done);
  p.pubq = reinterpret_cast<PubEntry*>(dc + L.off_pubq);
  p.tasks = reinterpret_cast<DevTask*>(dc + L.off_tasks);
  p.host_desc = reinterpret_cast<const TaskBody*>(dh + off_descs);
  p.host_heads = reinterpret_cast<const HostHead*>(dh + off_heads);
  p.host_complete = reinterpret_cast<HostComplete*>(dh + off_comp);
  p.host_shared = reinterpret_cast<HostShared*>(dh + off_shared);
  p.ranks = R;
  p.depth = D;
  p.qcap = L.qcap;
  p.quantum = (uint32_t)cfg.ingest_quantum;
  p.prefetch = cfg.l2_prefetch ? 1u : 0u;
  p.drain = 0;
  p.launch_gen = 0;
  p.wait_timeout_ns = cfg.wait_timeout_ns;
  p.idle_poll_ns = cfg.idle_poll_ns;

  // Copy streams the manager creates: one input and one output stream per
  // rank while they fit the stream budget with the scheduler's stream,
  // otherwise at most half of the budget each.
  const uint32_t budget = cfg.copy_streams_max > 0 ? (uint32_t)cfg.copy_streams_max : 31u;
  uint32_t n_in = R, n_out = R;
  if (cfg.copy_in_streams > 0) {
    n_in = std::min<uint32_t>(R, std::min<uint32_t>((uint32_t)cfg.copy_in_streams, budget > 1 ? budget - 1 : 1u));
    n_out = std::min<uint32_t>(R, std::max<uint32_t>(1u, budget - n_in));
  } else if (2 * R > budget) {
    n_in = std::min<uint32_t>(R, std::max<uint32_t>(1u, (budget + 1) / 2));
    n_out = std::min<uint32_t>(R, std::max<uint32_t>(1u, budget - n_in));
  }
  ctx->ranks.resize(R);
  for (uint32_t r = 0; r < R; ++r) {
    auto rk = std::make_unique<gvm_rank>();
    rk->ctx = ctx.get();
    rk->id = (int32_t)r;
    rk->slice = reinterpret_cast<uint64_t>(cfg.arena) + slice * r;
    rk->ring_base = rk->slice + resident;
    rk->ring_bytes = slice - resident;
    rk->slots.resize(D);
    if (cfg.copy_streams) {
      rk->in_stream = static_cast<cudaStream_t>(cfg.copy_streams[2 * r]);
      rk->out_stream = static_cast<cudaStream_t>(cfg.copy_streams[2 * r + 1]);
    } else {
      // Ranks beyond the stream budget share streams round robin (rank r
      // uses input stream r % n_in and output stream r % n_out).
      if (r < n_in) {
        e = cudaStreamCreateWithFlags(&rk->in_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) ctx->owned_streams.push_back(rk->in_stream);
      } else {
        rk->in_stream = ctx->ranks[r % n_in]->in_stream;
      }
      if (e == cudaSuccess && r < n_out) {
        e = cudaStreamCreateWithFlags(&rk->out_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) ctx->owned_streams.push_back(rk->out_stream);
      } else if (e == cudaSuccess) {
        rk->out_stream = ctx->ranks[r % n_out]->out_stream;
      }
      if (e != cudaSuccess) {
        cudaFreeHost(hb);
        return GVM_EDEVICE;
      }
    }
    ctx->ranks[r] = std::move(rk);
  }

  if (cfg.mode == GVM_MODE_CONTINUOUS) {
    // Resident until gvm_shutdown: launched before any output wait is pushed.
    std::lock_guard<std::mutex> g(ctx->launch_mu);
    int rc = launch_locked(ctx.get(), 0);
    if (rc != GVM_OK) {
      cudaFreeHost(hb);
      return rc;
    }
  }
  *out = ctx.release();
  return GVM_OK;
}

void* gvm_stream(gvm_ctx* ctx, int32_t which) {
  if (!ctx) return nullptr;
  if (which == -1) return ctx->sched;
  if (which < 0 || which >= 2 * ctx->cfg.max_ranks) return nullptr;
  gvm_rank* r = ctx->ranks[which / 2].get();
  return (which & 1) ? r->out_stream : r->in_stream;
}

int gvm_attach(gvm_ctx* ctx, int32_t rank, gvm_rank** out) {
  if (!ctx || !out) return GVM_EINVAL;
  if (ctx->shut) return GVM_ESTATE;
  if (rank < 0 || rank >= ctx->cfg.max_ranks) return GVM_EINVAL;
  gvm_rank* r = ctx->ranks[rank].get();
  std::lock_guard<std::mutex> g(r->mu);
  if (r->attached) return GVM_EBUSY;
  r->attached = true;
  *out = r;
  return GVM_OK;
}

}  // extern "C"

namespace {

// One validated task of a batch.
struct Prep {
  const gvm_task* t;
  bool resident;
  uint64_t c_direct;                   // device address of c when the kernel writes it there, else 0
  bool out_pageable;                   // c is pageable: copied out by the host after completion
  uint64_t bytes_a, bytes_b, bytes_c;  // operand bytes
  uint64_t sa, sb, sc;                 // staging bytes (256-aligned; 0 when resident)
};

// Shape, offset and pointer checks of one task (nothing is reserved).
int prep_task(gvm_rank* r, const gvm_task* t, Prep* p) {
  const bool resident = (t->flags & GVM_TASK_RESIDENT) != 0;
  int p_kc = 1;  // kind of the output buffer (host_kind)
  if (t->flags & ~GVM_TASK_RESIDENT) return GVM_EINVAL;
  uint64_t bytes_a = 0, bytes_b = 0, bytes_c = 0;
  if (t->type == GVM_TASK_VADD || t->type == GVM_TASK_VMUL) {
    if (t->n < 0 || t->n > (int64_t(1) << 34)) return GVM_EINVAL;
    if (t->type == GVM_TASK_VMUL && (t->k < 1 || t->k > 1024)) return GVM_EINVAL;
    bytes_a = bytes_b = bytes_c = 4ull * (uint64_t)t->n;
  } else if (t->type == GVM_TASK_SGEMM) {
    if (t->m < 1 || t->k < 1 || t->n < 1 || t->m > 32768 || t->k > 32768 || t->n > 32768) return GVM_EINVAL;
    bytes_a = 4ull * (uint64_t)t->m * (uint64_t)t->k;
    bytes_b = 4ull * (uint64_t)t->k * (uint64_t)t->n;
    bytes_c = 4ull * (uint64_t)t->m * (uint64_t)t->n;
  } else {
    return GVM_EINVAL;
  }
  const uint64_t res_bytes = r->ring_base - r->slice;
  if (resident) {
    const uint64_t al = t->type == GVM_TASK_SGEMM ? 16 : 4;  // VADD, VMUL: 4
    const uint64_t offs[3] = {t->a_off, t->b_off, t->c_off};
    const uint64_t lens[3] = {bytes_a, bytes_b, bytes_c};
    for (int i = 0; i < 3; ++i) {
      if (offs[i] % al) return GVM_EINVAL;
      if (offs[i] > res_bytes || lens[i] > res_bytes - offs[i]) return GVM_EINVAL;
    }
  } else if (bytes_c > 0) {
    if (!t->a || !t->b || !t->c) return GVM_EINVAL;
    const int ka = host_kind(t->a), kb = host_kind(t->b), kc = host_kind(t->c);
    if (ka < 0 || kb < 0 || kc < 0) return GVM_EINVAL;
    p_kc = kc;
  }
  p->t = t;
  p->resident = resident;
  p->bytes_a = bytes_a;
  p->bytes_b = bytes_b;
  p->bytes_c = bytes_c;
  p->c_direct = 0;
  p->out_pageable = !resident && bytes_c > 0 && p_kc == 0 && !stream_mode(r->ctx);
  if (!resident && bytes_c > 0 && p_kc == 1 && r->ctx->cfg.direct_output && !stream_mode(r->ctx)) {
    // The buffer's device mapping (the same address under unified addressing).
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, t->c) == cudaSuccess && at.devicePointer != nullptr)
      p->c_direct = reinterpret_cast<uint64_t>(at.devicePointer);
    else
      (void)cudaGetLastError();
  }
  p->sa = resident ? 0 : align_up(bytes_a, 256);
  p->sb = resident ? 0 : align_up(bytes_b, 256);
  p->sc = (resident || p->c_direct) ? 0 : align_up(bytes_c, 256);
  return GVM_OK;
}

// Staging bytes the ring would charge for `bytes` now (incl. the waste at the
// ring's end), or 0 when it has no room.
uint64_t stage_room(const gvm_rank* r, uint64_t bytes) {
  const uint64_t pos = r->ring_head, off = pos % r->ring_bytes;
  const uint64_t waste = off + bytes > r->ring_bytes ? r->ring_bytes - off : 0;
  if (pos + waste + bytes - r->ring_tail > r->ring_bytes) return 0;
  return waste + bytes;
}

void fill_body(gvm_ctx* ctx, gvm_rank* r, const Prep& p, uint64_t seq, uint64_t da, uint64_t db, uint64_t dc,
               TaskBody* body) {
  const gvm_task* t = p.t;
  const uint32_t D = (uint32_t)ctx->cfg.ring_depth;
  memset(body, 0, sizeof(*body));
  body->type = (uint32_t)t->type;
  body->rank = (uint32_t)r->id;
  body->slot = (uint32_t)(seq & (D - 1));
  body->tag = tag_of(seq);
  body->flags = p.resident         ? 0u
                : p.c_direct       ? (kFlagNeedsReady | kFlagDirectOut)
                : p.out_pageable   ? kFlagNeedsReady  // completes on the device; reap copies C out
                                   : (kFlagNeedsReady | kFlagNeedsD2H);
  body->a = da;
  body->b = db;
  body->c = dc;
  if (t->type == GVM_TASK_VADD || t->type == GVM_TASK_VMUL) {
    body->n = t->n;
    body->k = t->type == GVM_TASK_VMUL ? t->k : 0;  // products per element
    int64_t vt = ctx->cfg.vadd_tile;
    if (vt == 0) {
      vt = (t->n + ctx->grid - 1) / std::max(ctx->grid, 1);
      vt = (vt + 4095) / 4096 * 4096;
      vt = std::min<int64_t>(std::max<int64_t>(vt, kVaddTileMin), kVaddTileMax);
    }
    body->vadd_tile = vt;
    body->ntiles = (uint32_t)((t->n + vt - 1) / vt);
  } else {
    body->m = t->m;
    body->k = t->k;
    body->n = t->n;
    // Split3: fused tiles (the bf16 split happens in the tile itself),
    // 128 x 256 or, in the wide form, 256 x 256.
    const bool tiles128 = ctx->path == kPathSplit3 || ctx->path == kPathSplit3Tma;
    const int tm = tiles128 ? kTcM : ctx->path == kPathSplit3Wide ? 256 : kFmaTile;
    const int tn = tiles128 ? kTcN : ctx->path == kPathSplit3Wide ? 256 : kFmaTile;
    if (ctx->path != kPathFma) body->flags |= kFlagSplit3;
    // Wide tiles land A by TMA: the task's own map of A at its device address.
    if (ctx->path == kPathSplit3Wide &&
        encode_wide_a_map(reinterpret_cast<const float*>(da), t->m, t->k, &body->tmA) == CUDA_SUCCESS)
      body->flags |= kFlagTmA;
    // The TMA form lands A and B by TMA: the task's own maps of both.
    int b3 = 0;
    if (ctx->path == kPathSplit3Tma &&
        encode_tma_maps(reinterpret_cast<const float*>(da), reinterpret_cast<const float*>(db), t->m, t->n, t->k,
                        &body->tmA, &body->tmB, &b3) == CUDA_SUCCESS)
      body->flags |= kFlagTmA | kFlagTmB | (b3 ? kFlagTmB3 : 0u);
    body->tiles_m = (uint32_t)((t->m + tm - 1) / tm);
    body->tiles_n = (uint32_t)((t->n + tn - 1) / tn);
    body->ntiles = body->tiles_m * body->tiles_n;
  }
  body->nsplit = 0;
}

// Admits tasks[0 .. count-1] of rank r in order, as far as the ring and the
// staging space allow now. The batch's host-mode tasks share one staging
// region: all their inputs first, in order, then all their outputs, so that
// inputs (and outputs) the caller keeps in adjacent host buffers move in a
// few large copies. Returns the number admitted; when that is 0, *err says
// why (GVM_EAGAIN: not now; anything else: task 0 is invalid or can never
// fit). Caller holds r->mu.
int submit_batch(gvm_rank* r, const gvm_task* tasks, uint32_t count, uint64_t* first_seq, int* err) {
  gvm_ctx* ctx = r->ctx;
  *err = GVM_OK;
  if (!r->attached || ctx->shut) {
    *err = GVM_ESTATE;
    return 0;
  }
  bind_device(ctx);
  if (ld_acq(&ctx->shared->status)) {  // the scheduler stopped on an error: admit nothing
    *err = GVM_EDEVICE;
    return 0;
  }
  const uint32_t D = (uint32_t)ctx->cfg.ring_depth;
  reap(r);
  const uint64_t seq0 = r->next_seq;
  const uint32_t free_slots = (uint32_t)(D - (seq0 - r->synced));
  if (r->ring_head == r->ring_tail && r->ring_head % r->ring_bytes) {
    // Empty ring: restart at its beginning, so that a region as large as the
    // ring fits again.
    r->ring_head = r->ring_tail = align_up(r->ring_head, r->ring_bytes);
  }
  uint32_t n = std::min(count, free_slots);

  // ---- validate (stop before the first invalid task)
  std::vector<Prep> prep(n);
  for (uint32_t i = 0; i < n; ++i) {
    const int rc = prep_task(r, &tasks[i], &prep[i]);
    if (rc != GVM_OK) {
      if (i == 0) {
        *err = rc;
        return 0;
      }
      n = i;
      break;
    }
  }
  if (n == 0) {
    // No free slot: the first task must still be valid to say "not now".
    if (count > 0) {
      Prep p0;
      const int rc = prep_task(r, &tasks[0], &p0);
      *err = rc != GVM_OK ? rc : GVM_EAGAIN;
    }
    return 0;
  }

  // ---- staging: the longest prefix whose region fits the ring and the cap now
  const uint64_t cap = ctx->cfg.admission_cap_bytes;
  const uint64_t staged_now = ctx->staged.load();
  uint64_t need = 0, held = 0;
  uint32_t k = 0;
  for (; k < n; ++k) {
    const uint64_t add = prep[k].sa + prep[k].sb + prep[k].sc;
    if (add == 0) continue;
    const uint64_t h = stage_room(r, need + add);
    if (h == 0 || (cap && staged_now + h > cap)) break;
    need += add;
    held = h;
  }
  if (k == 0) {
    const uint64_t add = prep[0].sa + prep[0].sb + prep[0].sc;
    *err = (add > r->ring_bytes || (cap && add > cap)) ? GVM_ENOMEM : GVM_EAGAIN;
    GVM_TRACE("submit: rank %d refused (%d): needs %llu, ring head %llu tail %llu of %llu, synced %llu next %llu",
              r->id, *err, (unsigned long long)add, (unsigned long long)r->ring_head,
              (unsigned long long)r->ring_tail, (unsigned long long)r->ring_bytes, (unsigned long long)r->synced,
              (unsigned long long)r->next_seq);
    return 0;
  }
  uint64_t base = 0;
  if (need) {
    const uint64_t pos = r->ring_head + (held - need);  // skip the waste at the ring's end
    base = r->ring_base + (pos % r->ring_bytes);
    r->ring_head = pos + need;
    const uint64_t st = ctx->staged.fetch_add(held) + held;
    uint64_t pk = ctx->staged_peak.load();
    while (st > pk && !ctx->staged_peak.compare_exchange_weak(pk, st)) {
    }
  }
  uint64_t in_total = 0;
  for (uint32_t i = 0; i < k; ++i) in_total += prep[i].sa + prep[i].sb;

  // ---- descriptors; input copies gathered into runs
  std::vector<CopyRun> runs, pieces;
  std::vector<uint32_t> ready_after;  // per task: index of the run that completes its inputs
  ready_after.assign(k, 0);
  uint64_t in_off = 0, out_off = in_total, last_host = UINT64_MAX;
  for (uint32_t i = 0; i < k; ++i)
    if (prep[i].sa + prep[i].sb + prep[i].sc) last_host = i;
  uint64_t h2d = 0;
  for (uint32_t i = 0; i < k; ++i) {
    const Prep& p = prep[i];
    const gvm_task* t = p.t;
    const uint64_t seq = seq0 + i;
    const uint32_t slot = (uint32_t)(seq & (D - 1));
    const uint32_t idx = (uint32_t)r->id * D + slot;
    uint64_t da, db, dc;
    if (p.resident) {
      da = r->slice + t->a_off;
      db = r->slice + t->b_off;
      dc = r->slice + t->c_off;
    } else {
      da = base + in_off;
      db = da + p.sa;
      dc = p.c_direct ? p.c_direct : base + out_off;
      in_off += p.sa + p.sb;
      out_off += p.sc;
    }
    TaskBody body;
    fill_body(ctx, r, p, seq, da, db, dc, &body);
    memcpy(&ctx->descs[idx], &body, sizeof(body));
    SlotInfo& si = r->slots[slot];
    si.bytes = (i == last_host) ? held : 0;
    si.stage_end = r->ring_head;
    si.needs_out = !p.resident && !stream_mode(ctx) && !p.c_direct && !p.out_pageable;
    si.out_pageable = p.out_pageable;
    if (p.c_direct) ctx->d2h.fetch_add(p.bytes_c);  // written by the kernel
    si.c_host = t->c;
    si.c_dev = dc;
    si.c_bytes = p.resident ? 0 : p.bytes_c;
    si.host_io = !p.resident;
    si.a_host = t->a;
    si.b_host = t->b;
    si.a_dev = da;
    si.b_dev = db;
    si.a_bytes = p.resident ? 0 : p.bytes_a;
    si.b_bytes = p.resident ? 0 : p.bytes_b;
    if (!p.resident && !stream_mode(ctx)) {
      const uint64_t srcs_dst[2][3] = {{da, (uint64_t)(uintptr_t)t->a, p.bytes_a},
                                       {db, (uint64_t)(uintptr_t)t->b, p.bytes_b}};
      for (int j = 0; j < 2; ++j) {
        const uint64_t dst = srcs_dst[j][0], bytes = srcs_dst[j][2];
        const uint8_t* src = reinterpret_cast<const uint8_t*>(srcs_dst[j][1]);
        if (bytes == 0) continue;
        h2d += bytes;
        pieces.push_back(CopyRun{dst, src, bytes, 0, 1});
        if (!runs.empty()) {
          CopyRun& b = runs.back();
          if (b.dst + b.bytes == dst && b.src + b.bytes == src && b.bytes + bytes <= ctx->cfg.copy_run_bytes) {
            b.bytes += bytes;
            b.pieces += 1;
            continue;
          }
        }
        runs.push_back(CopyRun{dst, src, bytes, (uint32_t)pieces.size() - 1, 1});
      }
      ready_after[i] = runs.empty() ? 0 : (uint32_t)runs.size() - 1;
    }
  }

  // ---- input copies, each task's ready word after the run that ends its inputs
  // (PS-1 / PS-2: gvm_flush issues them)
  if (!stream_mode(ctx)) {
    const DriverApi* api = driver_api();
    size_t next_ready = 0;
    auto write_ready = [&](uint32_t upto_run) -> bool {
      for (; next_ready < k; ++next_ready) {
        const Prep& p = prep[next_ready];
        if (p.resident) continue;
        if (!runs.empty() && ready_after[next_ready] > upto_run) return true;
        const uint64_t seq = seq0 + next_ready;
        const uint32_t idx = (uint32_t)r->id * D + (uint32_t)(seq & (D - 1));
        const CUresult cr = api->write_value32(reinterpret_cast<CUstream>(r->in_stream),
                                               reinterpret_cast<CUdeviceptr>(ctx->params.ready + idx), tag_of(seq),
                                               CU_STREAM_WRITE_VALUE_DEFAULT);
        if (cr != CUDA_SUCCESS) {
          GVM_TRACE("submit: ready write for rank %d seq %llu failed (%d)", r->id, (unsigned long long)seq, (int)cr);
          return false;
        }
      }
      return true;
    };
    bool ok = true;
    for (uint32_t j = 0; ok && j < runs.size(); ++j) {
      const cudaError_t e = issue_run(runs[j], pieces, cudaMemcpyHostToDevice, r->in_stream);
      if (e != cudaSuccess)
        GVM_TRACE("submit: copy of %llu bytes to 0x%llx failed: %s", (unsigned long long)runs[j].bytes,
                  (unsigned long long)runs[j].dst, cudaGetErrorString(e));
      ok = e == cudaSuccess;
      if (ok) ok = write_ready(j);
    }
    if (ok) ok = write_ready(UINT32_MAX);
    if (!ok) {
      *err = GVM_EDEVICE;  // the manager is now unusable for this rank
      return 0;
    }
    ctx->h2d.fetch_add(h2d);
  }

  // ---- publish the batch
  __atomic_store_n(&ctx->heads[r->id].head, (uint32_t)(seq0 + k), __ATOMIC_RELEASE);
  r->next_seq = seq0 + k;
  r->published.store(seq0 + k, std::memory_order_release);
  ctx->submitted.fetch_add(k);
  if (first_seq) *first_seq = seq0;
  if (ctx->cfg.mode == GVM_MODE_CONTINUOUS) {
    // The resident scheduler was launched before any output wait was pushed.
    if (push_out_ops(r, r->next_seq) != GVM_OK) {
      *err = GVM_EDEVICE;
      return (int)k;
    }
  }
  return (int)k;
}

}  // namespace

extern "C" {

int gvm_submit(gvm_rank* r, const gvm_task* t, uint64_t* seq_out) {
  if (!r || !t) return GVM_EINVAL;
  std::lock_guard<std::mutex> g(r->mu);
  int err = GVM_OK;
  const int n = submit_batch(r, t, 1, seq_out, &err);
  if (n == 1) return err;
  return err != GVM_OK ? err : GVM_EAGAIN;
}

int gvm_submit_many(gvm_rank* r, const gvm_task* tasks, uint32_t count, uint64_t* first_seq) {
  if (!r || (!tasks && count)) return GVM_EINVAL;
  if (count == 0) return 0;
  std::lock_guard<std::mutex> g(r->mu);
  int err = GVM_OK;
  const int n = submit_batch(r, tasks, count, first_seq, &err);
  if (n == 0 && err != GVM_EAGAIN) return err;
  if (n > 0 && err == GVM_EDEVICE) return GVM_EDEVICE;
  return n;
}

int gvm_poll(gvm_rank* r, uint64_t seq) {
  if (!r) return GVM_EINVAL;
  std::lock_guard<std::mutex> g(r->mu);
  if (seq >= r->next_seq) return GVM_EINVAL;
  bind_device(r->ctx);
  if (push_flushed(r) != GVM_OK) return GVM_EDEVICE;
  reap(r);
  if (r->synced > seq) return 1;
  if (r->copy_failed) return GVM_EDEVICE;
  const uint32_t D = (uint32_t)r->ctx->cfg.ring_depth;
  const uint32_t idx = (uint32_t)r->id * D + (uint32_t)(seq & (D - 1));
  if (seq + D >= r->next_seq && ld_acq(&r->ctx->completes[idx].tag) == tag_of(seq)) return 1;
  if (ld_acq(&r->ctx->shared->status)) return GVM_EDEVICE;
  return 0;
}

int gvm_sync(gvm_rank* r, uint64_t seq) {
  if (!r) return GVM_EINVAL;
  gvm_ctx* ctx = r->ctx;
  std::unique_lock<std::mutex> g(r->mu);
  if (seq >= r->next_seq) return GVM_EINVAL;
  // Barrier, PS-1, PS-2 modes: a task submitted after the last gvm_flush
  // never runs until the next one.
  if (flush_mode(ctx) && seq >= r->flushed.load(std::memory_order_acquire)) return GVM_ESTATE;
  bind_device(ctx);
  if (push_flushed(r) != GVM_OK) return GVM_EDEVICE;
  uint64_t last = r->synced;
  uint64_t t_prog = now_ns(), t_query = t_prog;
  const uint64_t t_wait = t_prog;
  uint32_t spins = 0;
  while (true) {
    reap(r);
    if (r->synced > seq) return GVM_OK;
    if (r->copy_failed) return GVM_EDEVICE;
    if (ld_acq(&ctx->shared->status)) return GVM_EDEVICE;
    const uint64_t now = now_ns();
    if (r->synced != last) {
      last = r->synced;
      t_prog = now;
    } else if (now - t_prog > ctx->cfg.wait_timeout_ns + kHostGraceNs) {
      return GVM_ETIMEDOUT;
    }
    // A kernel that died without writing its status word shows up in the
    // stream's state; ask the driver rarely (every rank may be waiting here,
    // and driver calls from many threads serialise).
    if (now - t_query > kStreamQueryNs) {
      t_query = now;
      cudaError_t e = cudaStreamQuery(stream_mode(ctx) ? r->in_stream : ctx->sched);
      if (e != cudaSuccess && e != cudaErrorNotReady) return GVM_EDEVICE;
    }
    if ((++spins & 63) == 0) {
      g.unlock();
      // Spin (yielding) for the first kSyncSpinNs, then poll every
      // kSyncSleepNs: waits that outlast a whole launch leave the host's
      // cores to the threads that have work. Shorter waits spin, because a
      // sleeping waiter sees its completion late (measured: sleeping from
      // 200 us on made each 1 ms step of 16 ranks x 64 SGEMM 512^3 17 us
      // longer).
      if (now - t_wait > kSyncSpinNs)
        short_sleep(kSyncSleepNs);
      else
        std::this_thread::yield();
      g.lock();
    }
  }
}

int gvm_flush(gvm_ctx* ctx) {
  if (!ctx) return GVM_EINVAL;
  if (ctx->shut) return GVM_ESTATE;
  if (ctx->cfg.mode == GVM_MODE_CONTINUOUS) return GVM_OK;  // the scheduler is resident
  bind_device(ctx);
  std::lock_guard<std::mutex> g(ctx->launch_mu);
  if (stream_mode(ctx)) return ps_flush_locked(ctx);
  // Every task published before this point is drained by the launch below.
  std::vector<uint64_t> upto(ctx->ranks.size());
  for (size_t i = 0; i < ctx->ranks.size(); ++i) upto[i] = ctx->ranks[i]->published.load(std::memory_order_acquire);
  const int rc = launch_locked(ctx, 1);
  GVM_TRACE("flush: launch %u rc=%d", ctx->launch_gen, rc);
  if (rc != GVM_OK) return rc;
  for (size_t i = 0; i < ctx->ranks.size(); ++i) {
    uint64_t f = ctx->ranks[i]->flushed.load();
    while (f < upto[i] && !ctx->ranks[i]->flushed.compare_exchange_weak(f, upto[i])) {
    }
  }
  return GVM_OK;
}

int gvm_wait_idle(gvm_ctx* ctx) {
  if (!ctx) return GVM_EINVAL;
  bind_device(ctx);
  if (ctx->cfg.mode == GVM_MODE_BARRIER) {  // a resident scheduler only stops at shutdown
    const int rc = wait_scheduler(ctx);
    if (rc != GVM_OK) return rc;
  }
  for (auto& rk : ctx->ranks) {
    if (cudaStreamSynchronize(rk->in_stream) != cudaSuccess) return GVM_EDEVICE;
    if (cudaStreamSynchronize(rk->out_stream) != cudaSuccess) return GVM_EDEVICE;
  }
  return ld_acq(&ctx->shared->status) ? GVM_EDEVICE : GVM_OK;
}

static int rank_copy(gvm_rank* r, uint64_t off, void* host, uint64_t bytes, bool to_dev) {
  if (!r || (!host && bytes)) return GVM_EINVAL;
  const uint64_t res = r->ring_base - r->slice;
  if (off > res || bytes > res - off) return GVM_EINVAL;
  if (!bytes) return GVM_OK;
  bind_device(r->ctx);
  void* dev = reinterpret_cast<void*>(r->slice + off);
  cudaError_t e = to_dev ? cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, r->in_stream)
                         : cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, r->in_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(r->in_stream);
  return e == cudaSuccess ? GVM_OK : GVM_EDEVICE;
}

int gvm_rank_write(gvm_rank* r, uint64_t off, const void* src, uint64_t bytes) {
  return rank_copy(r, off, const_cast<void*>(src), bytes, true);
}

int gvm_rank_read(gvm_rank* r, uint64_t off, void* dst, uint64_t bytes) {
  return rank_copy(r, off, dst, bytes, false);
}

void* gvm_rank_resident_ptr(gvm_rank* r) { return r ? reinterpret_cast<void*>(r->slice) : nullptr; }

int gvm_detach(gvm_rank* r) {
  if (!r) return GVM_EINVAL;
  if (!r->attached) return GVM_ESTATE;
  if (flush_mode(r->ctx) && r->flushed.load() < r->published.load()) return GVM_ESTATE;
  if (r->next_seq > 0) {
    int rc = gvm_sync(r, r->next_seq - 1);
    if (rc != GVM_OK) return rc;
  }
  std::lock_guard<std::mutex> g(r->mu);
  r->attached = false;
  return GVM_OK;
}

int gvm_shutdown(gvm_ctx* ctx) {
  if (!ctx) return GVM_EINVAL;
  // A serving thread of gvm_ipc still drives this manager's ranks.
  if (ctx->ipc_servers.load(std::memory_order_acquire) > 0) return GVM_ESTATE;
  bind_device(ctx);
  int rc = GVM_OK;
  {
    std::lock_guard<std::mutex> g(ctx->launch_mu);
    if (ctx->shut) return GVM_ESTATE;
    ctx->shut = true;
    // Barrier mode: one last drain for tasks submitted since the last flush.
    bool pending = false;
    for (auto& rk : ctx->ranks)
      if (rk->flushed.load() < rk->published.load()) pending = true;
    if (ctx->cfg.mode == GVM_MODE_BARRIER && pending) {
      if (launch_locked(ctx, 1) != GVM_OK) rc = GVM_EDEVICE;
      for (auto& rk : ctx->ranks) rk->flushed.store(rk->published.load());
    } else if (stream_mode(ctx) && pending) {
      if (ps_flush_locked(ctx) != GVM_OK) rc = GVM_EDEVICE;
    }
  }
  GVM_TRACE("shutdown: stop (launches=%llu)", (unsigned long long)ctx->launches.load());
  // Continuous mode: the resident scheduler drains what is pending, then exits.
  __atomic_store_n(&ctx->shared->stop, 1u, __ATOMIC_RELEASE);
  for (auto& rk : ctx->ranks) {
    std::lock_guard<std::mutex> g(rk->mu);
    if (rc == GVM_OK && push_out_ops(rk.get(), rk->next_seq) != GVM_OK) rc = GVM_EDEVICE;
  }
  GVM_TRACE("shutdown: output ops pushed, waiting for the scheduler");
  const int wrc = wait_scheduler(ctx);
  if (wrc == GVM_ETIMEDOUT) {
    // The scheduler did not stop within the bound: leave the rings allocated
    // (the kernel may still read them) and report.
    return GVM_ETIMEDOUT;
  }
  if (wrc != GVM_OK) rc = wrc;
  const bool device_ok = ld_acq(&ctx->shared->status) == 0;
  GVM_TRACE("shutdown: scheduler idle, device_ok=%d", (int)device_ok);
  const DriverApi* api = driver_api();
  const uint32_t D = (uint32_t)ctx->cfg.ring_depth;
  for (auto& rk : ctx->ranks) {
    GVM_TRACE("shutdown: rank %d: input stream (out_pushed=%llu synced=%llu next=%llu)", rk->id,
              (unsigned long long)rk->out_pushed, (unsigned long long)rk->synced,
              (unsigned long long)rk->next_seq);
    if (cudaStreamSynchronize(rk->in_stream) != cudaSuccess) rc = GVM_EDEVICE;
    // An output stream still waiting after the scheduler has exited waits
    // for a done word no launch will write: wait a bounded time, then treat
    // it like a device error.
    bool out_stuck = false;
    if (device_ok) {
      const uint64_t t0 = now_ns();
      cudaError_t q;
      while ((q = cudaStreamQuery(rk->out_stream)) == cudaErrorNotReady &&
             now_ns() - t0 < ctx->cfg.wait_timeout_ns + kHostGraceNs)
        std::this_thread::yield();
      out_stuck = q == cudaErrorNotReady;
      if (out_stuck) {
        fprintf(stderr, "[gvm] shutdown: rank %d output stream still waits (synced=%llu out_pushed=%llu)\n", rk->id,
                (unsigned long long)rk->synced, (unsigned long long)rk->out_pushed);
        rc = GVM_ETIMEDOUT;
      }
    }
    if (!device_ok || out_stuck) {
      // The scheduler stopped on an error: release every output-stream wait
      // whose done word will never be written, so that the caller's streams
      // do not stay blocked after the manager is gone. Those tasks' outputs
      // are not valid.
      reap(rk.get());
      for (uint64_t s = rk->synced; s < rk->out_pushed; ++s) {
        const uint32_t idx = (uint32_t)rk->id * D + (uint32_t)(s & (D - 1));
        if (api->write_value32(reinterpret_cast<CUstream>(rk->in_stream),
                               reinterpret_cast<CUdeviceptr>(ctx->params.done + idx), tag_of(s),
                               CU_STREAM_WRITE_VALUE_DEFAULT) != CUDA_SUCCESS)
          rc = GVM_EDEVICE;
      }
      if (cudaStreamSynchronize(rk->in_stream) != cudaSuccess) rc = GVM_EDEVICE;
    }
    GVM_TRACE("shutdown: rank %d: output stream", rk->id);
    if (cudaStreamSynchronize(rk->out_stream) != cudaSuccess) rc = GVM_EDEVICE;
    GVM_TRACE("shutdown: rank %d streams idle (synced=%llu next=%llu)", rk->id, (unsigned long long)rk->synced,
              (unsigned long long)rk->next_seq);
  }
  if (!device_ok) rc = GVM_EDEVICE;
  GVM_TRACE("shutdown: freeing host rings");
  cudaFreeHost(ctx->host_block);
  delete ctx;
  return rc;
}

int gvm_stats_get(gvm_ctx* ctx, gvm_stats* out) {
  if (!ctx || !out) return GVM_EINVAL;
  out->submitted = ctx->submitted.load();
  out->completed = ctx->completed.load();
  out->launches = ctx->launches.load();
  out->staged_bytes = ctx->staged.load();
  out->staged_peak = ctx->staged_peak.load();
  out->h2d_bytes = ctx->h2d.load();
  out->d2h_bytes = ctx->d2h.load();
  out->device_status = ld_acq(&ctx->shared->status);
  out->device_where = ld_acq(&ctx->shared->where);
  out->launch_start_ns = __atomic_load_n(&ctx->shared->k_start, __ATOMIC_ACQUIRE);
  out->launch_last_done_ns = __atomic_load_n(&ctx->shared->k_last_done, __ATOMIC_ACQUIRE);
  out->launch_exit_ns = __atomic_load_n(&ctx->shared->k_exit, __ATOMIC_ACQUIRE);
  for (int i = 0; i < kProfSlots; ++i)
    out->launch_phase[i] = __atomic_load_n(&ctx->shared->k_prof[i], __ATOMIC_ACQUIRE);
  return GVM_OK;
}

int gvm_task_times(gvm_rank* r, uint64_t seq, uint64_t* t_ingest_ns, uint64_t* t_done_ns) {
  if (!r || !t_ingest_ns || !t_done_ns) return GVM_EINVAL;
  const uint32_t D = (uint32_t)r->ctx->cfg.ring_depth;
  if (seq >= r->next_seq || seq + D < r->next_seq) return GVM_EINVAL;
  const uint32_t idx = (uint32_t)r->id * D + (uint32_t)(seq & (D - 1));
  const HostComplete* hc = &r->ctx->completes[idx];
  if (ld_acq(&hc->tag) != tag_of(seq)) return GVM_ESTATE;
  *t_ingest_ns = __atomic_load_n(&hc->t_ingest, __ATOMIC_ACQUIRE);
  *t_done_ns = __atomic_load_n(&hc->t_done, __ATOMIC_ACQUIRE);
  return GVM_OK;
}

}  // extern "C"
