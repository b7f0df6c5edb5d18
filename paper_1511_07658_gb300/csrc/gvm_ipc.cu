// Cross-process ranks: POSIX shared-memory segments, one per rank, and the
// manager's serving thread (Section 5: SPMD processes reach the GVM through
// request/response queues and a shared data region). Host code only; the
// client functions make no CUDA call.
#include <cuda_runtime.h>
#include <errno.h>
#include <fcntl.h>
#include <signal.h>
#include <sys/mman.h>
#include <sys/stat.h>
#include <unistd.h>

#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "gvm_ipc.h"
#include "gvm_runtime.h"

namespace {

constexpr uint32_t kMagic = 0x47564d49u;  // "GVMI"
constexpr uint32_t kVersion = 1;
constexpr uint64_t kPage = 4096;
constexpr uint64_t kDataAlign = 2ull << 20;
constexpr uint64_t kLivenessNs = 100ull * 1000 * 1000;  // pid checks, both sides
constexpr uint32_t kBatch = 64;                          // requests per gvm_submit_many

static_assert(std::atomic<uint64_t>::is_always_lock_free, "64-bit atomics across processes");
static_assert(std::atomic<uint32_t>::is_always_lock_free, "32-bit atomics across processes");

// Header at the start of every segment. Counters are monotonic over the
// segment's life; each is written by one side only.
struct IpcShared {
  uint32_t magic, version;
  int32_t rank, nranks;
  uint32_t depth, pad0;
  uint64_t data_off, data_bytes;
  // written by the client
  alignas(64) std::atomic<uint64_t> head;         // requests written
  alignas(64) std::atomic<uint64_t> arrived;      // request-barrier arrivals
  std::atomic<uint64_t> arrive_head;              // head at the last arrival
  alignas(64) std::atomic<uint32_t> state;        // GVM_IPC_*
  std::atomic<int32_t> client_pid;
  // written by the manager
  alignas(64) std::atomic<uint64_t> tail;         // requests taken
  alignas(64) std::atomic<uint64_t> done;         // tasks complete, results in the data area
  alignas(64) std::atomic<int32_t> error;         // first refused or failed task: its code ...
  std::atomic<uint64_t> error_seq;                // ... and sequence number
  alignas(64) std::atomic<int32_t> server_pid;    // 0 while not served
  std::atomic<uint32_t> stopped;                  // the manager stopped serving
};

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

uint64_t align_up_u64(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

bool valid_name(const char* name) {
  if (!name) return false;
  const size_t n = strlen(name);
  if (n < 1 || n > 40) return false;
  for (size_t i = 0; i < n; ++i) {
    const char c = name[i];
    const bool ok = (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || (c >= '0' && c <= '9') || c == '_' ||
                    c == '-';
    if (!ok) return false;
  }
  return true;
}

std::string seg_name(const char* name, int32_t rank) { return "/" + std::string(name) + "." + std::to_string(rank); }

uint64_t ring_off() { return align_up_u64(sizeof(IpcShared), 64); }

uint64_t data_offset(uint32_t depth) { return align_up_u64(ring_off() + (uint64_t)depth * sizeof(gvm_ipc_task), kPage); }

gvm_ipc_task* ring_of(IpcShared* s) {
  return reinterpret_cast<gvm_ipc_task*>(reinterpret_cast<uint8_t*>(s) + ring_off());
}

// A process that exists and has not ended (a zombie, ended but not yet
// reaped by its parent, counts as ended).
bool pid_alive(int32_t pid) {
  if (pid <= 0) return false;
  if (kill(pid, 0) != 0 && errno != EPERM) return false;
  char path[64];
  snprintf(path, sizeof(path), "/proc/%d/stat", (int)pid);
  FILE* f = fopen(path, "r");
  if (!f) return true;
  char buf[512];
  const size_t n = fread(buf, 1, sizeof(buf) - 1, f);
  fclose(f);
  buf[n] = 0;
  const char* rp = strrchr(buf, ')');  // state follows the command name
  return !(rp && rp[1] == ' ' && (rp[2] == 'Z' || rp[2] == 'X'));
}

constexpr uint32_t kOpening = 4;  // transient: a client is taking the rank

struct Segment {
  IpcShared* s = nullptr;
  size_t map_bytes = 0;
  bool registered = false;  // data area page-locked by gvm_ipc_serve
};

}  // namespace

struct gvm_ipc_region {
  std::string name;
  int32_t nranks = 0;
  uint32_t depth = 0;
  uint64_t data_bytes = 0;
  std::vector<Segment> seg;
  bool served = false;
};

struct gvm_ipc_client {
  IpcShared* s = nullptr;
  size_t map_bytes = 0;
  uint64_t last_server_check = 0;
};

namespace {

// Manager-side state of one rank.
struct RankServe {
  gvm_rank* rank = nullptr;
  IpcShared* s = nullptr;
  uint8_t* data = nullptr;
  uint64_t taken = 0;     // requests consumed (submitted, or refused)
  uint64_t submitted = 0; // requests handed to gvm (== the gvm rank's next sequence number)
  uint64_t done = 0;      // tasks complete
  bool failed = false;    // a refused or failed task stopped this rank
  bool lost = false;
  // Request barrier: the client's arrivals covered by barriers run so far,
  // and the count taken when the current barrier opened (this rank in it).
  uint64_t arrivals_served = 0, arrivals_snap = 0;
  bool in_barrier = false;
};

}  // namespace

struct gvm_ipc_server {
  gvm_ctx* ctx = nullptr;
  gvm_ipc_region* region = nullptr;
  std::vector<RankServe> rs;
  std::thread th;
  std::atomic<bool> stop{false};
  std::atomic<uint64_t> taken{0}, completed{0}, barriers{0};
  bool barrier_open = false;
  int mode = GVM_MODE_BARRIER;
};

namespace {

void fail_rank(RankServe& r, int code, uint64_t seq) {
  r.failed = true;
  int32_t zero = 0;
  if (r.s->error.compare_exchange_strong(zero, code)) r.s->error_seq.store(seq, std::memory_order_release);
}

// Offsets and sizes of one request against the rank's data area; fills the
// gvm_task with host pointers into it.
int to_task(const RankServe& r, const gvm_ipc_task& q, gvm_task* t) {
  if (q.reserved != 0) return GVM_EINVAL;
  uint64_t la = 0, lb = 0, lc = 0;
  if (q.type == GVM_TASK_VADD || q.type == GVM_TASK_VMUL) {
    if (q.n < 0 || q.n > (int64_t(1) << 34)) return GVM_EINVAL;
    la = lb = lc = 4ull * (uint64_t)q.n;
  } else if (q.type == GVM_TASK_SGEMM) {
    if (q.m < 1 || q.n < 1 || q.k < 1 || q.m > 32768 || q.n > 32768 || q.k > 32768) return GVM_EINVAL;
    la = 4ull * (uint64_t)q.m * (uint64_t)q.k;
    lb = 4ull * (uint64_t)q.k * (uint64_t)q.n;
    lc = 4ull * (uint64_t)q.m * (uint64_t)q.n;
  } else {
    return GVM_EINVAL;
  }
  const uint64_t cap = r.s->data_bytes;
  const uint64_t offs[3] = {q.a_off, q.b_off, q.c_off}, lens[3] = {la, lb, lc};
  for (int i = 0; i < 3; ++i)
    if (offs[i] > cap || lens[i] > cap - offs[i]) return GVM_EINVAL;
  memset(t, 0, sizeof(*t));
  t->type = q.type;
  t->flags = 0;
  t->m = q.m;
  t->n = q.n;
  t->k = q.k;
  t->a = r.data + q.a_off;
  t->b = r.data + q.b_off;
  t->c = r.data + q.c_off;
  return GVM_OK;
}

// Takes the rank's new requests into the manager, as far as it admits them
// now. Returns true if anything moved.
bool ingest(gvm_ipc_server* sv, RankServe& r) {
  const uint64_t head = r.s->head.load(std::memory_order_acquire);
  bool moved = false;
  const gvm_ipc_task* ring = ring_of(r.s);
  const uint32_t D = r.s->depth;
  while (r.taken < head) {
    if (r.failed) {  // everything after a refused task is dropped
      r.taken = head;
      r.s->tail.store(r.taken, std::memory_order_release);
      return true;
    }
    gvm_task batch[kBatch];
    uint32_t cnt = 0;
    int bad = GVM_OK;
    while (cnt < kBatch && r.taken + cnt < head) {
      const gvm_ipc_task q = ring[(r.taken + cnt) & (D - 1)];
      bad = to_task(r, q, &batch[cnt]);
      if (bad != GVM_OK) break;
      ++cnt;
    }
    if (cnt > 0) {
      uint64_t first = 0;
      const int n = gvm_submit_many(r.rank, batch, cnt, &first);
      if (n < 0) {
        fail_rank(r, n, r.taken);
        continue;
      }
      if (n == 0) break;  // the rank's staging or ring is full: later
      r.taken += (uint64_t)n;
      r.submitted += (uint64_t)n;
      sv->taken.fetch_add((uint64_t)n);
      r.s->tail.store(r.taken, std::memory_order_release);
      moved = true;
      if ((uint32_t)n < cnt) break;
      continue;
    }
    // The next request is invalid: refuse it; the rank stops there.
    fail_rank(r, bad, r.taken);
    r.taken += 1;
    r.s->tail.store(r.taken, std::memory_order_release);
    moved = true;
  }
  return moved;
}

// Publishes completions in order. Returns true if anything moved.
bool reap_done(RankServe& r) {
  bool moved = false;
  while (r.done < r.submitted) {
    const int p = gvm_poll(r.rank, r.done);
    if (p == 1) {
      ++r.done;
      moved = true;
      continue;
    }
    if (p < 0) fail_rank(r, p, r.done);
    break;
  }
  if (moved) r.s->done.store(r.done, std::memory_order_release);
  return moved;
}

bool attached(const RankServe& r) {
  return !r.lost && r.s->state.load(std::memory_order_acquire) == GVM_IPC_ATTACHED;
}

void serve_loop(gvm_ipc_server* sv) {
  const bool flush_mode = sv->mode != GVM_MODE_CONTINUOUS;
  uint64_t last_live = now_ns();
  uint32_t idle = 0;
  uint64_t flushed_upto = 0;  // sum of submitted counts covered by the last flush
  while (!sv->stop.load(std::memory_order_acquire)) {
    bool moved = false;
    uint64_t total_sub = 0;
    for (auto& r : sv->rs) {
      moved |= ingest(sv, r);
      total_sub += r.submitted;
    }
    // Request barrier (flush modes): it opens once every attached client
    // has an arrival not yet served (clients that attach later join the
    // next one), then flushes until each of them has every request up to
    // its arrival taken.
    if (flush_mode) {
      if (!sv->barrier_open) {
        bool any = false, all = true;
        for (auto& r : sv->rs) {
          if (!attached(r)) continue;
          any = true;
          if (r.s->arrived.load(std::memory_order_acquire) <= r.arrivals_served) all = false;
        }
        if (any && all) {
          sv->barrier_open = true;
          for (auto& r : sv->rs) {
            r.in_barrier = attached(r);
            if (r.in_barrier) r.arrivals_snap = r.s->arrived.load(std::memory_order_acquire);
          }
        }
      }
      if (sv->barrier_open) {
        if (total_sub > flushed_upto) {
          if (gvm_flush(sv->ctx) != GVM_OK) {
            for (auto& r : sv->rs) fail_rank(r, GVM_EDEVICE, r.done);
          }
          flushed_upto = total_sub;
          moved = true;
        }
        bool complete = true;
        for (auto& r : sv->rs) {
          if (!r.in_barrier || !attached(r) || r.failed) continue;
          if (r.taken < r.s->arrive_head.load(std::memory_order_acquire)) complete = false;
        }
        if (complete) {
          for (auto& r : sv->rs) {
            if (r.in_barrier) r.arrivals_served = r.arrivals_snap;
            r.in_barrier = false;
          }
          sv->barriers.fetch_add(1);
          sv->barrier_open = false;
        }
      }
    }
    uint64_t comp = 0;
    for (auto& r : sv->rs) {
      moved |= reap_done(r);
      comp += r.done;
    }
    sv->completed.store(comp);
    // Liveness of the clients: a process that ended without closing leaves
    // the barrier (its taken tasks still run).
    const uint64_t t = now_ns();
    if (t - last_live > kLivenessNs) {
      last_live = t;
      for (auto& r : sv->rs) {
        if (r.s->state.load(std::memory_order_acquire) != GVM_IPC_ATTACHED) continue;
        if (!pid_alive(r.s->client_pid.load())) {
          uint32_t exp = GVM_IPC_ATTACHED;
          r.s->state.compare_exchange_strong(exp, GVM_IPC_LOST);
        }
      }
    }
    if (moved) {
      idle = 0;
    } else if (++idle < 256) {
      std::this_thread::yield();
    } else {
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
}

int map_segment(int fd, size_t bytes, IpcShared** out) {
  void* p = mmap(nullptr, bytes, PROT_READ | PROT_WRITE, MAP_SHARED, fd, 0);
  if (p == MAP_FAILED) return GVM_ENOMEM;
  *out = static_cast<IpcShared*>(p);
  return GVM_OK;
}

}  // namespace

extern "C" {

int gvm_ipc_create(const char* name, int32_t nranks, uint64_t data_bytes, int32_t depth, gvm_ipc_region** out) {
  if (!out || !valid_name(name) || nranks < 1 || nranks > GVM_MAX_RANKS || data_bytes == 0 ||
      data_bytes > (1ull << 40) || depth < 2 || depth > 4096 || (depth & (depth - 1)))
    return GVM_EINVAL;
  *out = nullptr;
  auto reg = new gvm_ipc_region();
  reg->name = name;
  reg->nranks = nranks;
  reg->depth = (uint32_t)depth;
  reg->data_bytes = align_up_u64(data_bytes, kDataAlign);
  const uint64_t doff = data_offset(reg->depth);
  const size_t total = (size_t)(doff + reg->data_bytes);
  int rc = GVM_OK;
  for (int32_t r = 0; r < nranks && rc == GVM_OK; ++r) {
    const std::string sn = seg_name(name, r);
    const int fd = shm_open(sn.c_str(), O_RDWR | O_CREAT | O_EXCL, 0600);
    if (fd < 0) {
      rc = errno == EEXIST ? GVM_EBUSY : GVM_EINVAL;
      break;
    }
    // Reserve every page now: a shared-memory file system too small for the
    // region fails here instead of faulting a process later.
    if (ftruncate(fd, (off_t)total) != 0 || posix_fallocate(fd, 0, (off_t)total) != 0) {
      close(fd);
      shm_unlink(sn.c_str());
      rc = GVM_ENOMEM;
      break;
    }
    Segment sg;
    sg.map_bytes = total;
    rc = map_segment(fd, total, &sg.s);
    close(fd);
    if (rc != GVM_OK) {
      shm_unlink(sn.c_str());
      break;
    }
    IpcShared* s = sg.s;
    memset(static_cast<void*>(s), 0, (size_t)doff);  // counters start at 0
    s->magic = kMagic;
    s->version = kVersion;
    s->rank = r;
    s->nranks = nranks;
    s->depth = reg->depth;
    s->data_off = doff;
    s->data_bytes = reg->data_bytes;
    s->state.store(GVM_IPC_FREE, std::memory_order_release);
    reg->seg.push_back(sg);
  }
  if (rc != GVM_OK) {
    for (size_t r = 0; r < reg->seg.size(); ++r) {
      munmap(reg->seg[r].s, reg->seg[r].map_bytes);
      shm_unlink(seg_name(name, (int32_t)r).c_str());
    }
    delete reg;
    return rc;
  }
  *out = reg;
  return GVM_OK;
}

int gvm_ipc_destroy(gvm_ipc_region* reg) {
  if (!reg) return GVM_EINVAL;
  if (reg->served) return GVM_ESTATE;
  int rc = GVM_OK;
  for (size_t r = 0; r < reg->seg.size(); ++r) {
    Segment& sg = reg->seg[r];
    if (sg.registered) {
      IpcShared* s = sg.s;
      if (cudaHostUnregister(reinterpret_cast<uint8_t*>(s) + s->data_off) != cudaSuccess) {
        (void)cudaGetLastError();
        rc = GVM_EDEVICE;
      }
      sg.registered = false;
    }
    munmap(reg->seg[r].s, reg->seg[r].map_bytes);
    shm_unlink(seg_name(reg->name.c_str(), (int32_t)r).c_str());
  }
  delete reg;
  return rc;
}

int gvm_ipc_peek(gvm_ipc_region* reg, int32_t rank, uint64_t* head, uint64_t* arrived, uint64_t* done,
                 uint32_t* state) {
  if (!reg || rank < 0 || rank >= reg->nranks) return GVM_EINVAL;
  IpcShared* s = reg->seg[rank].s;
  if (head) *head = s->head.load(std::memory_order_acquire);
  if (arrived) *arrived = s->arrived.load(std::memory_order_acquire);
  if (done) *done = s->done.load(std::memory_order_acquire);
  if (state) *state = s->state.load(std::memory_order_acquire);
  return GVM_OK;
}

int gvm_ipc_serve(gvm_ctx* ctx, gvm_ipc_region* reg, gvm_ipc_server** out) {
  if (!ctx || !reg || !out) return GVM_EINVAL;
  if (reg->served) return GVM_ESTATE;
  if (reg->nranks > gvm::ctx_max_ranks(ctx)) return GVM_EINVAL;
  *out = nullptr;
  auto sv = new gvm_ipc_server();
  sv->ctx = ctx;
  sv->region = reg;
  sv->mode = gvm::ctx_mode(ctx);
  sv->rs.resize((size_t)reg->nranks);
  int rc = GVM_OK;
  for (int32_t r = 0; r < reg->nranks && rc == GVM_OK; ++r) {
    RankServe& rs = sv->rs[r];
    rs.s = reg->seg[r].s;
    rs.data = reinterpret_cast<uint8_t*>(rs.s) + rs.s->data_off;
    // Counters continue from the segment's past (a region may be served
    // again); the gvm rank starts at sequence 0, so only a fresh segment maps
    // request numbers onto gvm sequence numbers one to one.
    if (rs.s->head.load() != 0 || rs.s->tail.load() != 0) {
      rc = GVM_ESTATE;
      break;
    }
    // Page-locked once per region; gvm_ipc_destroy releases it (after the
    // manager has shut down: a resident scheduler holds the device until then).
    if (!reg->seg[r].registered) {
      if (cudaHostRegister(rs.data, (size_t)rs.s->data_bytes,
                                         cudaHostRegisterPortable | cudaHostRegisterMapped) != cudaSuccess) {
        (void)cudaGetLastError();
        rc = GVM_EDEVICE;
        break;
      }
      reg->seg[r].registered = true;
    }
    rc = gvm_attach(ctx, r, &rs.rank);
  }
  if (rc != GVM_OK) {
    for (auto& rs : sv->rs)
      if (rs.rank) gvm_detach(rs.rank);
    delete sv;
    return rc;
  }
  const int32_t pid = (int32_t)getpid();
  for (auto& rs : sv->rs) {
    rs.s->stopped.store(0, std::memory_order_release);
    rs.s->server_pid.store(pid, std::memory_order_release);
  }
  reg->served = true;
  gvm::ctx_servers_add(ctx, 1);
  sv->th = std::thread(serve_loop, sv);
  *out = sv;
  return GVM_OK;
}

int gvm_ipc_stop(gvm_ipc_server* sv) {
  if (!sv) return GVM_EINVAL;
  sv->stop.store(true, std::memory_order_release);
  if (sv->th.joinable()) sv->th.join();
  int rc = GVM_OK;
  // A last barrier for what was taken, then wait for it.
  if (sv->mode != GVM_MODE_CONTINUOUS) {
    const int f = gvm_flush(sv->ctx);
    if (f != GVM_OK) rc = f;
  }
  for (auto& r : sv->rs) {
    if (r.submitted > r.done) {
      const int s = gvm_sync(r.rank, r.submitted - 1);
      if (s == GVM_OK) {
        r.done = r.submitted;
      } else {
        fail_rank(r, s, r.done);
        if (rc == GVM_OK) rc = s;
      }
    }
    r.s->done.store(r.done, std::memory_order_release);
    r.s->stopped.store(1, std::memory_order_release);
    r.s->server_pid.store(0, std::memory_order_release);
  }
  for (auto& r : sv->rs) {
    const int d = gvm_detach(r.rank);
    if (d != GVM_OK && rc == GVM_OK) rc = d;
  }
  sv->region->served = false;
  gvm::ctx_servers_add(sv->ctx, -1);
  delete sv;
  return rc;
}

int gvm_ipc_server_counts(gvm_ipc_server* sv, uint64_t* taken, uint64_t* completed, uint64_t* barriers) {
  if (!sv) return GVM_EINVAL;
  if (taken) *taken = sv->taken.load();
  if (completed) *completed = sv->completed.load();
  if (barriers) *barriers = sv->barriers.load();
  return GVM_OK;
}

// ---- client side ----------------------------------------------------------

int gvm_ipc_open(const char* name, int32_t rank, gvm_ipc_client** out) {
  if (!out || !valid_name(name) || rank < 0) return GVM_EINVAL;
  *out = nullptr;
  const std::string sn = seg_name(name, rank);
  const int fd = shm_open(sn.c_str(), O_RDWR, 0600);
  if (fd < 0) return GVM_EINVAL;
  struct stat st;
  if (fstat(fd, &st) != 0 || (uint64_t)st.st_size < sizeof(IpcShared)) {
    close(fd);
    return GVM_EINVAL;
  }
  IpcShared* s = nullptr;
  const int rc = map_segment(fd, (size_t)st.st_size, &s);
  close(fd);
  if (rc != GVM_OK) return rc;
  if (s->magic != kMagic || s->version != kVersion || s->rank != rank ||
      s->data_off + s->data_bytes > (uint64_t)st.st_size) {
    munmap(s, (size_t)st.st_size);
    return GVM_EINVAL;
  }
  // Take the rank: free, closed or lost; or held by a process that has ended.
  // The transient state keeps a second opener out while the pid is written.
  uint32_t cur = s->state.load(std::memory_order_acquire);
  for (;;) {
    if (cur == kOpening || (cur == GVM_IPC_ATTACHED && pid_alive(s->client_pid.load()))) {
      munmap(s, (size_t)st.st_size);
      return GVM_EBUSY;
    }
    if (s->state.compare_exchange_weak(cur, kOpening, std::memory_order_acq_rel)) break;
  }
  s->client_pid.store((int32_t)getpid(), std::memory_order_release);
  s->state.store(GVM_IPC_ATTACHED, std::memory_order_release);
  auto c = new gvm_ipc_client();
  c->s = s;
  c->map_bytes = (size_t)st.st_size;
  *out = c;
  return GVM_OK;
}

void* gvm_ipc_data(gvm_ipc_client* c, uint64_t* bytes) {
  if (!c) return nullptr;
  if (bytes) *bytes = c->s->data_bytes;
  return reinterpret_cast<uint8_t*>(c->s) + c->s->data_off;
}

int gvm_ipc_submit(gvm_ipc_client* c, const gvm_ipc_task* t, uint64_t* seq) {
  if (!c || !t) return GVM_EINVAL;
  IpcShared* s = c->s;
  if (s->stopped.load(std::memory_order_acquire)) return GVM_ECANCELED;
  const uint64_t h = s->head.load(std::memory_order_relaxed);
  if (h - s->tail.load(std::memory_order_acquire) >= s->depth) return GVM_EAGAIN;
  ring_of(s)[h & (s->depth - 1)] = *t;
  s->head.store(h + 1, std::memory_order_release);
  if (seq) *seq = h;
  return GVM_OK;
}

int gvm_ipc_barrier(gvm_ipc_client* c) {
  if (!c) return GVM_EINVAL;
  IpcShared* s = c->s;
  s->arrive_head.store(s->head.load(std::memory_order_relaxed), std::memory_order_release);
  s->arrived.fetch_add(1, std::memory_order_acq_rel);
  return GVM_OK;
}

int gvm_ipc_wait(gvm_ipc_client* c, uint64_t seq, uint64_t timeout_ns) {
  if (!c) return GVM_EINVAL;
  IpcShared* s = c->s;
  if (seq >= s->head.load(std::memory_order_relaxed)) return GVM_EINVAL;
  const uint64_t t0 = now_ns();
  uint32_t spins = 0;
  for (;;) {
    if (s->done.load(std::memory_order_acquire) > seq) return GVM_OK;
    const int32_t e = s->error.load(std::memory_order_acquire);
    if (e != 0 && seq >= s->error_seq.load(std::memory_order_acquire)) return e;
    if (s->stopped.load(std::memory_order_acquire)) {
      return s->done.load(std::memory_order_acquire) > seq ? GVM_OK : GVM_ECANCELED;
    }
    const uint64_t t = now_ns();
    if (timeout_ns && t - t0 > timeout_ns) return GVM_ETIMEDOUT;
    if (t - c->last_server_check > kLivenessNs) {
      c->last_server_check = t;
      const int32_t sp = s->server_pid.load(std::memory_order_acquire);
      if (sp != 0 && !pid_alive(sp)) return GVM_ECANCELED;
    }
    // Spin briefly, then back off: many clients may wait at once on as many
    // cores as the manager's serving thread needs.
    if (++spins > 4096) {
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    } else if (spins > 64) {
      std::this_thread::yield();
    }
  }
}

int gvm_ipc_close(gvm_ipc_client* c) {
  if (!c) return GVM_EINVAL;
  c->s->state.store(GVM_IPC_CLOSED, std::memory_order_release);
  munmap(c->s, c->map_bytes);
  delete c;
  return GVM_OK;
}

}  // extern "C"
