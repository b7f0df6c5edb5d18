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
constexpr uint64_t kHostGraceNs = 1000ull * 1000 * 1000;

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
  int device = 0;
  std::vector<cudaStream_t> owned_streams;  // created by gvm_init, destroyed by gvm_shutdown
  ~gvm_ctx() {
    for (cudaStream_t st : owned_streams) cudaStreamDestroy(st);
  }
};

namespace {

bool cfg_valid(const gvm_config* c) {
  if (!c) return false;
  if (c->max_ranks < 1 || c->max_ranks > GVM_MAX_RANKS) return false;
  if (c->ring_depth < 2 || c->ring_depth > 4096 || (c->ring_depth & (c->ring_depth - 1))) return false;
  if (c->mode != GVM_MODE_BARRIER && c->mode != GVM_MODE_CONTINUOUS) return false;
  if (c->sgemm_path != GVM_SGEMM_FMA && c->sgemm_path != GVM_SGEMM_SPLIT3) return false;
  return true;
}

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
    if (si.bytes) {
      r->ring_tail = si.stage_end;
      ctx->staged.fetch_sub(si.bytes);
      si.bytes = 0;
    }
    r->synced = s + 1;
    ctx->completed.fetch_add(1);
  }
}

// Reserve `bytes` (a multiple of 256) in the rank's staging ring. Returns the
// device address, 0 when there is no room right now. *held gets the bytes
// charged (including any space skipped at the ring's end).
uint64_t stage_alloc(gvm_rank* r, uint64_t bytes, uint64_t* held) {
  if (bytes == 0) {
    *held = 0;
    return 0;
  }
  uint64_t pos = r->ring_head;
  const uint64_t off = pos % r->ring_bytes;
  uint64_t waste = 0;
  if (off + bytes > r->ring_bytes) waste = r->ring_bytes - off;
  if (pos + waste + bytes - r->ring_tail > r->ring_bytes) return 0;
  pos += waste;
  r->ring_head = pos + bytes;
  *held = waste + bytes;
  return r->ring_base + (pos % r->ring_bytes);
}

// Pushes the output operations (wait on done, device-to-host copy, completion
// word) of tasks out_pushed .. upto-1 on the rank's output stream. Called only
// once the scheduler launch that will write those done words has been pushed:
// a blocked wait can then never sit ahead of its own producer in a hardware
// queue that two streams share.
int push_out_ops(gvm_rank* r, uint64_t upto) {
  gvm_ctx* ctx = r->ctx;
  const DriverApi* api = driver_api();
  const uint32_t D = (uint32_t)ctx->cfg.ring_depth;
  while (r->out_pushed < upto) {
    const uint64_t s = r->out_pushed;
    SlotInfo& si = r->slots[s & (D - 1)];
    if (si.needs_out) {
      const uint32_t idx = (uint32_t)r->id * D + (uint32_t)(s & (D - 1));
      const uint32_t tag = tag_of(s);
      CUresult cr = api->wait_value32(reinterpret_cast<CUstream>(r->out_stream),
                                      reinterpret_cast<CUdeviceptr>(ctx->params.done + idx), tag,
                                      CU_STREAM_WAIT_VALUE_EQ);
      cudaError_t e = cudaSuccess;
      if (cr == CUDA_SUCCESS && si.c_bytes)
        e = cudaMemcpyAsync(si.c_host, reinterpret_cast<void*>(si.c_dev), si.c_bytes, cudaMemcpyDeviceToHost,
                            r->out_stream);
      if (cr == CUDA_SUCCESS && e == cudaSuccess)
        cr = api->write_value32(reinterpret_cast<CUstream>(r->out_stream),
                                reinterpret_cast<CUdeviceptr>(&ctx->params.host_complete[idx].tag), tag,
                                CU_STREAM_WRITE_VALUE_DEFAULT);
      if (cr != CUDA_SUCCESS || e != cudaSuccess) return GVM_EDEVICE;
      ctx->d2h.fetch_add(si.c_bytes);
      si.needs_out = false;
    }
    r->out_pushed = s + 1;
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

bool is_pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
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
  ctx->path = cfg.sgemm_path == GVM_SGEMM_SPLIT3 ? kPathSplit3 : kPathFma;
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
  p.drain = 0;
  p.launch_gen = 0;
  p.wait_timeout_ns = cfg.wait_timeout_ns;
  p.idle_poll_ns = cfg.idle_poll_ns;

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
      e = cudaStreamCreateWithFlags(&rk->in_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess) ctx->owned_streams.push_back(rk->in_stream);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&rk->out_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess) ctx->owned_streams.push_back(rk->out_stream);
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

int gvm_submit(gvm_rank* r, const gvm_task* t, uint64_t* seq_out) {
  if (!r || !t) return GVM_EINVAL;
  gvm_ctx* ctx = r->ctx;
  std::lock_guard<std::mutex> g(r->mu);
  if (!r->attached || ctx->shut) return GVM_ESTATE;
  bind_device(ctx);
  const bool resident = (t->flags & GVM_TASK_RESIDENT) != 0;
  if (t->flags & ~GVM_TASK_RESIDENT) return GVM_EINVAL;
  const bool split3 = ctx->path == kPathSplit3;

  // ---- shape and operand checks
  uint64_t bytes_a = 0, bytes_b = 0, bytes_c = 0;
  if (t->type == GVM_TASK_VADD) {
    if (t->n < 0 || t->n > (int64_t(1) << 34)) return GVM_EINVAL;
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
    const uint64_t al = t->type == GVM_TASK_SGEMM ? 16 : 4;
    const uint64_t offs[3] = {t->a_off, t->b_off, t->c_off};
    const uint64_t lens[3] = {bytes_a, bytes_b, bytes_c};
    for (int i = 0; i < 3; ++i) {
      if (offs[i] % al) return GVM_EINVAL;
      if (offs[i] > res_bytes || lens[i] > res_bytes - offs[i]) return GVM_EINVAL;
    }
  } else if (bytes_c > 0) {
    if (!t->a || !t->b || !t->c) return GVM_EINVAL;
    if (!is_pinned(t->a) || !is_pinned(t->b) || !is_pinned(t->c)) return GVM_EINVAL;
  }

  const uint32_t D = (uint32_t)ctx->cfg.ring_depth;
  reap(r);
  const uint64_t seq = r->next_seq;
  if (seq - r->synced >= D) return GVM_EAGAIN;

  // ---- staging: copied operands (host mode)
  const uint64_t sa = resident ? 0 : align_up(bytes_a, 256);
  const uint64_t sb = resident ? 0 : align_up(bytes_b, 256);
  const uint64_t sc = resident ? 0 : align_up(bytes_c, 256);
  const uint64_t need = sa + sb + sc;
  if (need > r->ring_bytes) return GVM_ENOMEM;
  const uint64_t cap = ctx->cfg.admission_cap_bytes;
  if (cap && need > cap) return GVM_ENOMEM;
  if (cap && ctx->staged.load() + need > cap) return GVM_EAGAIN;
  uint64_t held = 0, base = 0;
  if (need) {
    base = stage_alloc(r, need, &held);
    if (!base) return GVM_EAGAIN;
  }
  const uint64_t st = ctx->staged.fetch_add(held) + held;
  uint64_t pk = ctx->staged_peak.load();
  while (st > pk && !ctx->staged_peak.compare_exchange_weak(pk, st)) {
  }
  SlotInfo& si = r->slots[seq & (D - 1)];
  si.bytes = held;
  si.stage_end = r->ring_head;

  // ---- descriptor
  const uint32_t slot = (uint32_t)(seq & (D - 1));
  const uint32_t idx = (uint32_t)r->id * D + slot;
  const uint32_t tag = tag_of(seq);
  TaskBody body;
  memset(&body, 0, sizeof(body));
  body.type = (uint32_t)t->type;
  body.rank = (uint32_t)r->id;
  body.slot = slot;
  body.tag = tag;
  body.flags = resident ? 0u : (kFlagNeedsReady | kFlagNeedsD2H);
  uint64_t da, db, dcp;
  if (resident) {
    da = r->slice + t->a_off;
    db = r->slice + t->b_off;
    dcp = r->slice + t->c_off;
  } else {
    da = base;
    db = base + sa;
    dcp = base + sa + sb;
  }
  body.a = da;
  body.b = db;
  body.c = dcp;
  if (t->type == GVM_TASK_VADD) {
    body.n = t->n;
    int64_t vt = (t->n + ctx->grid - 1) / std::max(ctx->grid, 1);
    vt = (vt + 4095) / 4096 * 4096;
    vt = std::min<int64_t>(std::max<int64_t>(vt, kVaddTileMin), kVaddTileMax);
    body.vadd_tile = vt;
    body.ntiles = (uint32_t)((t->n + vt - 1) / vt);
    body.nsplit = 0;
  } else {
    body.m = t->m;
    body.k = t->k;
    body.n = t->n;
    if (split3) {
      // Fused split3 tiles (the bf16 split happens in the tile itself).
      body.flags |= kFlagSplit3;
      body.tiles_m = (uint32_t)((t->m + kTcM - 1) / kTcM);
      body.tiles_n = (uint32_t)((t->n + kTcN - 1) / kTcN);
      body.nsplit = 0;
      body.ntiles = body.tiles_m * body.tiles_n;
    } else {
      body.tiles_m = (uint32_t)((t->m + kFmaTile - 1) / kFmaTile);
      body.tiles_n = (uint32_t)((t->n + kFmaTile - 1) / kFmaTile);
      body.nsplit = 0;
      body.ntiles = body.tiles_m * body.tiles_n;
    }
  }
  memcpy(&ctx->descs[idx], &body, sizeof(body));

  // ---- host mode: input copies + ready; output wait + copy + completion
  if (!resident) {
    const DriverApi* api = driver_api();
    cudaError_t e = cudaSuccess;
    if (bytes_a) e = cudaMemcpyAsync(reinterpret_cast<void*>(da), t->a, bytes_a, cudaMemcpyHostToDevice, r->in_stream);
    if (e == cudaSuccess && bytes_b)
      e = cudaMemcpyAsync(reinterpret_cast<void*>(db), t->b, bytes_b, cudaMemcpyHostToDevice, r->in_stream);
    CUresult cr = CUDA_SUCCESS;
    if (e == cudaSuccess)
      cr = api->write_value32(reinterpret_cast<CUstream>(r->in_stream),
                              reinterpret_cast<CUdeviceptr>(ctx->params.ready + idx), tag,
                              CU_STREAM_WRITE_VALUE_DEFAULT);
    if (e != cudaSuccess || cr != CUDA_SUCCESS) return GVM_EDEVICE;  // manager now unusable for this rank
    ctx->h2d.fetch_add(bytes_a + bytes_b);
    si.c_host = t->c;
    si.c_dev = dcp;
    si.c_bytes = bytes_c;
    si.needs_out = true;
  } else {
    si.needs_out = false;
  }

  // ---- publish
  __atomic_store_n(&ctx->heads[r->id].head, (uint32_t)(seq + 1), __ATOMIC_RELEASE);
  r->next_seq = seq + 1;
  r->published.store(seq + 1, std::memory_order_release);
  ctx->submitted.fetch_add(1);
  if (seq_out) *seq_out = seq;
  if (ctx->cfg.mode == GVM_MODE_CONTINUOUS) {
    // The resident scheduler was launched before any output wait was pushed.
    return push_out_ops(r, r->next_seq);
  }
  return GVM_OK;
}

int gvm_submit_many(gvm_rank* r, const gvm_task* tasks, uint32_t count, uint64_t* first_seq) {
  if (!r || (!tasks && count)) return GVM_EINVAL;
  uint32_t done = 0;
  for (; done < count; ++done) {
    uint64_t s = 0;
    const int rc = gvm_submit(r, &tasks[done], &s);
    if (rc != GVM_OK) {
      if (done == 0 && rc != GVM_EAGAIN) return rc;
      break;
    }
    if (done == 0 && first_seq) *first_seq = s;
  }
  return (int)done;
}

int gvm_poll(gvm_rank* r, uint64_t seq) {
  if (!r) return GVM_EINVAL;
  std::lock_guard<std::mutex> g(r->mu);
  if (seq >= r->next_seq) return GVM_EINVAL;
  bind_device(r->ctx);
  if (push_flushed(r) != GVM_OK) return GVM_EDEVICE;
  reap(r);
  if (r->synced > seq) return 1;
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
  // Barrier mode: a task submitted after the last gvm_flush never runs
  // until the next one.
  if (ctx->cfg.mode == GVM_MODE_BARRIER && seq >= r->flushed.load(std::memory_order_acquire))
    return GVM_ESTATE;
  bind_device(ctx);
  if (push_flushed(r) != GVM_OK) return GVM_EDEVICE;
  uint64_t last = r->synced;
  uint64_t t_prog = now_ns(), t_query = t_prog;
  uint32_t spins = 0;
  while (true) {
    reap(r);
    if (r->synced > seq) return GVM_OK;
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
      cudaError_t e = cudaStreamQuery(ctx->sched);
      if (e != cudaSuccess && e != cudaErrorNotReady) return GVM_EDEVICE;
    }
    if ((++spins & 63) == 0) {
      g.unlock();
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
  if (r->ctx->cfg.mode == GVM_MODE_BARRIER && r->flushed.load() < r->published.load()) return GVM_ESTATE;
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
    if (cudaStreamSynchronize(rk->in_stream) != cudaSuccess) rc = GVM_EDEVICE;
    if (!device_ok) {
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
