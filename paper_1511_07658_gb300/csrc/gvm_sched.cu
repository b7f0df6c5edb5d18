// Persistent scheduler of the GPU virtualization manager.
//
// The paper's manager (Section 5) is a daemon that owns the only GPU context,
// takes requests from per-process queues, waits at a request barrier and
// flushes every process's stream so that kernels and copies of different
// processes overlap (Section 4.2.2). Here the request queues are rings of task
// descriptors in pinned host memory, one per rank, and the manager's request
// loop is this kernel: its CTAs take descriptors from the rings (round robin
// over ranks, FIFO within a rank), cut each task into tiles, and run tiles of
// all ranks' tasks side by side -- the concurrency the paper gets from one
// stream per process, without a kernel launch per task.
//
// Work flow per CTA:
//   claim:   every queue entry covers a contiguous range of one global tile
//            space; a CTA takes the next tile index with one atomicAdd on
//            next_tile and finds its entry by a short forward search. An
//            index beyond the published tiles is a reservation the CTA waits
//            for (ingesting meanwhile). Warp 0 claims the next tile while the
//            other warps run the current one.
//   ingest:  one CTA at a time (holding a lock) copies ready descriptors from
//            the host rings into the device task table and appends queue
//            entries (split phases of a pass before main phases, so the
//            split3 pre-pass of a task runs well ahead of its GEMM).
//   finish:  the CTA that completes a task's last tile publishes completion:
//            the host completion word (resident tasks) or the device done word
//            on which the rank's output-copy stream waits (host-buffer tasks).
//
// Every wait is bounded (wait_timeout_ns); a wait that runs out records a
// status word in host memory and stops the kernel. In continuous mode the
// kernel stays resident until the host sets the stop word (idle CTAs sleep
// idle_poll_ns between polls); in barrier (drain) mode it exits once every
// descriptor published before its launch has been taken.
#include "gvm_device.cuh"
#include <cstddef>
#include <type_traits>

#include "gvm_fused.cuh"
#include "gvm_runtime.h"
#include "gvm_tma.cuh"
#include "gvm_wide.cuh"

namespace gvm {

// FMA path: two tile slots; the CTA runs the tile in one while warp 0 claims
// the next into the other. go: 1 = a tile is there, 0 = exit, 2 = nothing
// claimed yet.
struct alignas(128) SchedShared {
  TaskBody body[2];  // copies of the claimed tasks' bodies
  uint32_t go[2];
  uint32_t task[2];
  uint32_t phase[2];
  uint32_t tile[2];
  uint32_t need[2];  // per iteration parity: a blocking claim must follow the tile
  uint32_t abort;
  uint32_t fail_where;
  uint64_t prof[kProfSlots];  // this CTA's phase counters (kProf*), written by thread 0 only
  uint64_t claim[4];  // Claim state (see acquire), owned by warp 0
};

constexpr uint32_t kMaxQuantum = 8;
constexpr uint64_t kLookaheadTiles = 512;  // ingest ahead when this few published tiles remain
constexpr uint64_t kQuietNs = 20000; // skip look-ahead ingest this long after an empty pass

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

__device__ void report_error(const SchedParams& p, uint32_t status, uint32_t where, uint32_t info) {
  HostShared* hs = p.host_shared;
  *reinterpret_cast<volatile uint32_t*>(&hs->where) = where;
  *reinterpret_cast<volatile uint32_t*>(&hs->info) = info;
  __threadfence_system();
  st_release_sys(&hs->status, status);
  atomicExch(&p.ctrl->abort, 1u);
}

// Marks task idx complete: timestamps, then the word its waiter watches.
__device__ void complete_task(const SchedParams& p, uint32_t idx, uint32_t tag, uint32_t flags,
                              uint64_t t_ingest) {
  HostComplete* hc = &p.host_complete[idx];
  const uint64_t now = globaltimer();
  st_relaxed_sys64(&hc->t_ingest, t_ingest);
  st_relaxed_sys64(&hc->t_done, now);
  atomicMax(reinterpret_cast<unsigned long long*>(&p.ctrl->t_last_done), (unsigned long long)now);
  __threadfence_system();
  if (flags & kFlagNeedsD2H) {
    st_release_sys(&p.done[idx], tag);
  } else {
    st_release_sys(&hc->tag, tag);
  }
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

struct IngestOut {
  uint32_t locked_out;
  uint32_t published;
  uint32_t pending;
};

// Warp 0 of one CTA: move ready descriptors from the host rings into the
// device table and append their queue entries, each covering a contiguous
// range of the global tile space. All lanes call.
template <bool kPrefetch>
__device__ IngestOut ingest(const SchedParams& p, uint64_t* prof) {
  const int lane = threadIdx.x & 31;
  IngestOut out{0, 0, 0};
  uint32_t got = 0;
  if (lane == 0) got = (atomicCAS(&p.ctrl->ingest_lock, 0u, 1u) == 0u) ? 1u : 0u;
  got = __shfl_sync(0xffffffffu, got, 0);
  if (!got) {
    out.locked_out = 1;
    return out;
  }
  __threadfence();
  // Drain mode: once a pass has found the rings empty (`drained`, set below
  // under this lock), nothing more is published in this launch, even if the
  // host has published descriptors since: CTAs leave with reservations
  // beyond the published tiles, and a tile published after its reserver
  // left would never run. Those descriptors wait in the rings for the next
  // launch.
  uint32_t closed = 0;
  if (lane == 0 && p.drain) closed = ld_relaxed_gpu(&p.ctrl->drained);
  if (__shfl_sync(0xffffffffu, closed, 0)) {
    if (lane == 0) {
      __threadfence();
      atomicExch(&p.ctrl->ingest_lock, 0u);
    }
    __syncwarp();
    return out;
  }
  const uint64_t pub0 = ld_relaxed_gpu64(&p.ctrl->published);
  const uint64_t tiles0 = ld_relaxed_gpu64(&p.ctrl->published_tiles);
  const uint64_t consumed = ld_relaxed_gpu64(&p.ctrl->cursor);
  const uint32_t rr = ld_relaxed_gpu(&p.ctrl->rr);
  const uint64_t now = globaltimer();
  uint64_t pub = pub0, ptiles = tiles0;
  uint32_t pending = 0;
  bool bad = false;

  for (uint32_t g = 0; g < p.ranks; g += 32) {
    // Keep at most half the ring between the hand-out frontier and the
    // newest entry, so that an entry is read long before its slot is reused.
    const uint64_t used = pub - consumed;
    const uint32_t space = used < p.qcap / 2 ? (uint32_t)(p.qcap / 2 - used) : 0u;
    uint32_t quantum = min(p.quantum, kMaxQuantum);
    // Each task takes at most two queue entries.
    const uint32_t lanes = min(32u, p.ranks - g);
    if (2u * lanes * quantum > space) quantum = space / (2u * lanes);

    uint32_t r = 0, t = 0, take = 0, avail = 0;
    uint32_t tidx[kMaxQuantum], tsplit[kMaxQuantum], tmain[kMaxQuantum];
    uint32_t nsplit_e = 0, nmain_e = 0, split_tiles = 0, main_tiles = 0;
    const bool valid = (g + lane) < p.ranks;
    if (valid) {
      r = (rr + g + lane) % p.ranks;
      const uint32_t h = ld_acquire_sys(&p.host_heads[r].head);
      t = ld_relaxed_gpu(&p.tail[r]);
      avail = h - t;
      const uint32_t lim = min(avail, quantum);
      // The task fields are the descriptor's last 128 bytes (its first 256, the
      // pre-pass form's tensor maps, are not used here). One read of them from
      // host memory gives both the readiness rule and the fields to copy.
      constexpr int kFieldsAt = offsetof(TaskBody, type) / 16;
      static_assert(offsetof(TaskBody, type) == 256 && sizeof(TaskBody) == 384, "TaskBody fields");
      static_assert(offsetof(TaskBody, flags) == 260 && offsetof(TaskBody, tag) == 272 &&
                        offsetof(TaskBody, ntiles) == 276 && offsetof(TaskBody, nsplit) == 280,
                    "TaskBody header words");
      // kPrefetch: descriptor s + 1 is read while s is processed, so that a
      // lane's host round trips overlap instead of following one another
      // (32 more registers; the FMA scheduler, which would spill, reads them
      // one by one).
      auto fields_of = [&](uint32_t s) {
        return reinterpret_cast<const uint4*>(&p.host_desc[r * p.depth + (s & (p.depth - 1))]) + kFieldsAt;
      };
      uint4 vn[kPrefetch ? 8 : 1];
      if (kPrefetch && lim > 0) {
        const uint4* src = fields_of(t);
#pragma unroll
        for (int j = 0; j < 8; ++j) vn[kPrefetch ? j : 0] = ld_volatile_v4(src + j);
      }
      for (; take < lim; ++take) {
        const uint32_t s = t + take;
        const uint32_t idx = r * p.depth + (s & (p.depth - 1));
        uint4 v[8];
        if constexpr (kPrefetch) {
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = vn[j];
          if (take + 1 < lim) {
            const uint4* nsrc = fields_of(s + 1);
#pragma unroll
            for (int j = 0; j < 8; ++j) vn[j] = ld_volatile_v4(nsrc + j);
          }
        } else {
          const uint4* src = fields_of(s);
#pragma unroll
          for (int j = 0; j < 8; ++j) v[j] = ld_volatile_v4(src + j);
        }
        const uint32_t flags = v[0].y;
        if ((flags & kFlagNeedsReady) && ld_acquire_gpu(&p.ready[idx]) != s + 1u) break;
        DevTask* dt = &p.tasks[idx];
        uint4* dst = reinterpret_cast<uint4*>(&dt->body) + kFieldsAt;
#pragma unroll
        for (int j = 0; j < 8; ++j) st_cg_v4(dst + j, v[j]);
        if (flags & (kFlagTmA | kFlagTmB)) {  // the tensor maps (the descriptor's first 128 or 256 bytes)
          static_assert(offsetof(TaskBody, tmA) == 0 && offsetof(TaskBody, tmB) == 128 &&
                            sizeof(CUtensorMap) == 128, "TaskBody maps");
          const uint4* m_src = reinterpret_cast<const uint4*>(&p.host_desc[idx]);
          uint4* m_dst = reinterpret_cast<uint4*>(&dt->body);
          const int nv = (flags & kFlagTmB) ? 16 : 8;
#pragma unroll 1
          for (int j = 0; j < nv; ++j) st_cg_v4(m_dst + j, ld_volatile_v4(m_src + j));
        }
        const uint32_t tag = v[1].x;
        const uint32_t ntiles = v[1].y;
        const uint32_t nsplit = v[1].z;
        tidx[take] = idx;
        tsplit[take] = tmain[take] = 0;
        if (tag != s + 1u || nsplit > ntiles) {
          bad = true;
          continue;
        }
        atomicExch(&dt->tiles_done, 0u);
        atomicExch(&dt->split_done, 0u);
        *reinterpret_cast<volatile uint64_t*>(&dt->t_ingest) = now;
        if (ntiles == 0) {
          __threadfence();
          complete_task(p, idx, tag, flags, now);
          continue;
        }
        tsplit[take] = nsplit;
        tmain[take] = ntiles - nsplit;
        if (nsplit) {
          ++nsplit_e;
          split_tiles += nsplit;
        }
        if (ntiles > nsplit) {
          ++nmain_e;
          main_tiles += ntiles - nsplit;
        }
      }
    }

    // Split entries of this pass first, then main entries, each group in lane
    // order: the split3 pre-pass of a task is handed out well ahead of its GEMM.
    const uint32_t ie_s = warp_incl_scan(nsplit_e), ie_m = warp_incl_scan(nmain_e);
    const uint32_t it_s = warp_incl_scan(split_tiles), it_m = warp_incl_scan(main_tiles);
    const uint32_t te_s = __shfl_sync(0xffffffffu, ie_s, 31), te_m = __shfl_sync(0xffffffffu, ie_m, 31);
    const uint32_t tt_s = __shfl_sync(0xffffffffu, it_s, 31), tt_m = __shfl_sync(0xffffffffu, it_m, 31);
    uint64_t es = pub + ie_s - nsplit_e, em = pub + te_s + ie_m - nmain_e;
    uint64_t bs = ptiles + it_s - split_tiles, bm = ptiles + tt_s + it_m - main_tiles;
    for (uint32_t i = 0; i < take; ++i) {
      if (tsplit[i]) {
        PubEntry e{bs, es, tidx[i], kPhaseSplit, tsplit[i], 0};
        p.pubq[es & (p.qcap - 1)] = e;
        ++es;
        bs += tsplit[i];
      }
      if (tmain[i]) {
        PubEntry e{bm, em, tidx[i], kPhaseMain, tmain[i], 0};
        p.pubq[em & (p.qcap - 1)] = e;
        ++em;
        bm += tmain[i];
      }
    }
    if (valid && take > 0) *reinterpret_cast<volatile uint32_t*>(&p.tail[r]) = t + take;
    pending += avail - take;
    pub += te_s + te_m;
    ptiles += tt_s + tt_m;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) pending += __shfl_xor_sync(0xffffffffu, pending, d);
  const uint32_t any_bad = __any_sync(0xffffffffu, bad);
  __threadfence();
  fence_tensormap_release();
  __syncwarp();
  if (lane == 0) {
    if (pending == 0 && pub == pub0) {
      *reinterpret_cast<volatile uint64_t*>(&p.ctrl->quiet_until) = now + kQuietNs;
      if (p.drain) st_release_gpu(&p.ctrl->drained, 1u);  // under the lock: no later pass publishes
    }
    if (pub != pub0) {
      st_release_gpu64(&p.ctrl->published, pub);
      st_release_gpu64(&p.ctrl->published_tiles, ptiles);
    }
    *reinterpret_cast<volatile uint32_t*>(&p.ctrl->rr) = (rr + 1) % p.ranks;
    __threadfence();
    atomicExch(&p.ctrl->ingest_lock, 0u);
    if (any_bad) report_error(p, kStatusBadTask, 0, 0);
  }
  __syncwarp();
  out.published = (uint32_t)(pub - pub0);
  out.pending = pending;
  if (lane == 0 && out.published) {
    prof[kProfIngest] += globaltimer() - now;
    prof[kProfIngests] += 1;
  }
  return out;
}

__device__ __forceinline__ uint32_t bcast(uint32_t v) { return __shfl_sync(0xffffffffu, v, 0); }
__device__ __forceinline__ uint64_t bcast64(uint64_t v) {
  const uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)v, 0);
  const uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(v >> 32), 0);
  return ((uint64_t)hi << 32) | lo;
}

// A CTA's claim state, kept in shared memory across calls: a tile index
// handed out by next_tile that may lie beyond the published tiles (then the
// CTA waits for it, ingesting meanwhile), and where its entry search resumes.
struct Claim {
  uint64_t resv;     // reserved tile index
  uint64_t hint;     // queue entry to start the next search at
  uint64_t stall_since;  // when published descriptors started waiting for their inputs (0: not waiting)
  uint32_t has_resv;
  uint32_t pad;
};

// One warp: find the next tile to run. Returns 1 with (task, phase, tile) set,
// 0 when the kernel should exit, and 2 when the reserved tile is not
// published yet and either !blocking or a blocking call has found nothing for
// idle_return_ns (0: never). Decisions use values lane 0 read and broadcast,
// so the warp never diverges across the shuffles.
//
// Claiming is one atomicAdd on next_tile per tile: there is no per-entry
// counter for all CTAs to contend on. A tile beyond published_tiles is a
// reservation; tiles are published in increasing order, so it becomes valid
// without further claims.
template <bool kPrefetch>
__device__ int acquire(const SchedParams& p, Claim* cl, uint32_t& task, uint32_t& phase, uint32_t& tile,
                       uint64_t* prof, bool blocking, uint64_t idle_return_ns = 0) {
  const int lane = threadIdx.x & 31;
  uint64_t entered = 0;
  auto set_stall = [&](uint64_t v) {
    if (lane == 0) cl->stall_since = v;
    __syncwarp();
  };
  while (true) {
    uint32_t abort = 0, drained = 0;
    uint64_t pt = 0, npub = 0, now = 0, quiet = 0, x = 0;
    if (lane == 0) {
      abort = ld_relaxed_gpu(&p.ctrl->abort);
      drained = ld_acquire_gpu(&p.ctrl->drained);
      if (!cl->has_resv) {
        cl->resv = atomicAdd(reinterpret_cast<unsigned long long*>(&p.ctrl->next_tile), 1ull);
        cl->has_resv = 1;
      }
      x = cl->resv;
      pt = ld_acquire_gpu64(&p.ctrl->published_tiles);
      // Entries below `published` are complete: an ingest pass releases
      // `published` (before published_tiles) only after writing them. An
      // entry beyond it may be half written (new seq, old count).
      npub = ld_acquire_gpu64(&p.ctrl->published);
      quiet = ld_relaxed_gpu64(&p.ctrl->quiet_until);
      now = globaltimer();
    }
    if (bcast(abort)) return 0;
    drained = bcast(drained);
    if (entered == 0) entered = bcast64(now);
    x = bcast64(x);
    pt = bcast64(pt);
    npub = bcast64(npub);
    now = bcast64(now);
    quiet = bcast64(quiet);
    if (x < pt) {
      // Keep the queue ahead of the CTAs.
      if (pt - x <= kLookaheadTiles && now >= quiet) (void)ingest<kPrefetch>(p, prof);
      // Find the entry holding tile x: the last entry with base <= x. Entries
      // are published in tile order, and x only grows from one claim of a CTA
      // to the next, so the search starts at the entry of this CTA's previous
      // tile; the warp checks 32 entries per step.
      uint32_t etask = 0, ephase = 0, off = 0, ok = 1;
      uint64_t e0 = 0;
      if (lane == 0) e0 = cl->hint;
      e0 = bcast64(e0);
      while (true) {
        const uint64_t e = e0 + (uint64_t)lane;
        const PubEntry* pe = &p.pubq[e & (p.qcap - 1)];
        const uint64_t seq = ld_relaxed_gpu64(&pe->seq);
        const uint64_t base = ld_relaxed_gpu64(&pe->base);
        const bool le = (e < npub) && (seq == e) && base <= x;
        const uint32_t m = __ballot_sync(0xffffffffu, le);
        if (m == 0) {  // not even the first entry starts at or before x
          ok = 0;
          break;
        }
        const int last = 31 - __clz(m);
        if (last == 31 && (m & 1u)) {  // the whole window precedes x: move on
          e0 += 31;
          continue;
        }
        const uint32_t cnt = ld_relaxed_gpu(&pe->cnt);
        const uint32_t tk = ld_relaxed_gpu(&pe->task);
        const uint32_t ph = ld_relaxed_gpu(&pe->phase);
        const uint64_t hit_base = __shfl_sync(0xffffffffu, base, last);
        const uint32_t hit_cnt = __shfl_sync(0xffffffffu, cnt, last);
        etask = __shfl_sync(0xffffffffu, tk, last);
        ephase = __shfl_sync(0xffffffffu, ph, last) & 1u;
        if (x >= hit_base + hit_cnt) {  // a hole in the tile space: the ring bound was broken
          ok = 0;
          break;
        }
        off = (uint32_t)(x - hit_base);
        if (lane == 0) {
          const uint64_t ehit = e0 + (uint64_t)last;
          if (x + 1 == hit_base + hit_cnt)
            atomicMax(reinterpret_cast<unsigned long long*>(&p.ctrl->cursor), (unsigned long long)(ehit + 1));
          cl->hint = ehit;
          cl->has_resv = 0;
          cl->stall_since = 0;
        }
        __syncwarp();
        break;
      }
      if (!bcast(ok)) {
        if (lane == 0) report_error(p, kStatusBadTask, kWhereQueueFull, (uint32_t)x);
        __syncwarp();
        return 0;
      }
      task = bcast(etask);
      phase = bcast(ephase);
      tile = bcast(off);
      return 1;
    }
    // The reserved tile is not published yet. Before leaving, look at the
    // published tiles once more: another CTA's last ingest pass may have
    // published the reserved tile since pt was read, and a tile whose owner
    // leaves would never run. Once the rings are drained (or stop is set with
    // nothing pending) no further tile is published, so this read is final.
    auto reserved_published = [&]() -> bool {
      uint64_t pt2 = 0;
      if (lane == 0) pt2 = ld_acquire_gpu64(&p.ctrl->published_tiles);
      return x < bcast64(pt2);
    };
    if (p.drain && drained) {
      if (reserved_published()) continue;
      return 0;
    }
    const IngestOut r = ingest<kPrefetch>(p, prof);
    if (r.published) {
      set_stall(0);
      continue;
    }
    if (!r.locked_out) {
      if (r.pending == 0) {
        set_stall(0);
        if (p.drain) {  // this pass (or an earlier one) closed the launch: `drained` is set
          if (reserved_published()) continue;
          return 0;
        }
        uint32_t stop = 0;
        if (lane == 0) stop = ld_acquire_sys(&p.host_shared->stop);
        if (bcast(stop)) {
          if (reserved_published()) continue;
          return 0;
        }
      } else if (blocking) {
        uint64_t since = 0;
        if (lane == 0) {
          if (cl->stall_since == 0) cl->stall_since = now;
          since = cl->stall_since;
        }
        since = bcast64(since);
        if (now - since > p.wait_timeout_ns) {
          if (lane == 0) report_error(p, kStatusTimeout, kWhereReadyWait, r.pending);
          __syncwarp();
          return 0;
        }
      }
    }
    // Nothing to run yet. A look-ahead claim (made while the CTA still works
    // on its current tile) must not wait: the current tile's completion is
    // published only after it returns. The reservation is kept.
    if (!blocking) return 2;
    if (idle_return_ns != 0 && now - entered > idle_return_ns) return 2;
    __nanosleep(r.locked_out ? 200u : (uint32_t)p.idle_poll_ns);
  }
}

// Kernel entry bookkeeping: the launch's start time is the earliest CTA's.
__device__ void sched_enter(const SchedParams& p) {
  const unsigned long long t0 = globaltimer();
  unsigned long long* ts = reinterpret_cast<unsigned long long*>(&p.ctrl->t_start);
  if (atomicCAS(ts, 0ull, t0) != 0ull) atomicMin(ts, t0);
}

// Thread 0 of a CTA that is done: adds its phase counters; the last CTA of the
// launch publishes the launch's timeline and counters and resets the
// per-launch words for the next launch.
__device__ void sched_exit(const SchedParams& p, const uint64_t* prof) {
  for (int i = 0; i < kProfSlots; ++i)
    atomicAdd(reinterpret_cast<unsigned long long*>(&p.ctrl->prof[i]), (unsigned long long)prof[i]);
  __threadfence();
  const uint32_t n = atomicAdd(&p.ctrl->exit_count, 1u);
  if (n + 1 != gridDim.x) return;
  HostShared* hs = p.host_shared;
  st_relaxed_sys64(&hs->k_start, atomicExch(reinterpret_cast<unsigned long long*>(&p.ctrl->t_start), 0ull));
  st_relaxed_sys64(&hs->k_last_done,
                   atomicExch(reinterpret_cast<unsigned long long*>(&p.ctrl->t_last_done), 0ull));
  for (int i = 0; i < kProfSlots; ++i)
    st_relaxed_sys64(&hs->k_prof[i], atomicExch(reinterpret_cast<unsigned long long*>(&p.ctrl->prof[i]), 0ull));
  st_relaxed_sys64(&hs->k_exit, globaltimer());
  // Reservations beyond the published tiles died with their CTAs; the next
  // launch hands out tiles of entries published from here on.
  atomicExch(reinterpret_cast<unsigned long long*>(&p.ctrl->next_tile),
             (unsigned long long)ld_relaxed_gpu64(&p.ctrl->published_tiles));
  atomicExch(reinterpret_cast<unsigned long long*>(&p.ctrl->first_entry),
             (unsigned long long)ld_relaxed_gpu64(&p.ctrl->published));
  atomicExch(&p.ctrl->exit_count, 0u);
  atomicExch(&p.ctrl->drained, 0u);
  atomicExch(&p.ctrl->ingest_lock, 0u);
  __threadfence_system();
  st_release_sys(&p.host_shared->exit_gen, p.launch_gen);
}

// One tile of a task has finished (its results are visible device-wide):
// count it, and complete the task after its last tile.
__device__ void finish_tile(const SchedParams& p, uint32_t task, uint32_t ntiles, uint32_t tag, uint32_t flags) {
  DevTask* dt = &p.tasks[task];
  const uint32_t d = atomicAdd(&dt->tiles_done, 1u);
  if (d + 1 == ntiles) {
    __threadfence();
    const uint64_t t_in = *reinterpret_cast<volatile uint64_t*>(&dt->t_ingest);
    complete_task(p, task, tag, flags, t_in);
  }
}

// ------------------------------------------------------------ FMA scheduler

__global__ void __launch_bounds__(kThreads, 2) sched_fma_kernel(const SchedParams p) {
  __shared__ SchedShared sh;
  extern __shared__ uint8_t dyn_smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    sh.abort = 0;
    sh.fail_where = 0;
    for (int i = 0; i < kProfSlots; ++i) sh.prof[i] = 0;
    sched_enter(p);
  }
  Claim* cl = reinterpret_cast<Claim*>(sh.claim);
  if (tid == 0) {
    cl->has_resv = 0;
    cl->stall_since = 0;
    // Tiles handed out by this launch lie in entries published after it began
    // (a CTA may start after others of the launch have already published).
    cl->hint = ld_relaxed_gpu64(&p.ctrl->first_entry);
  }
  __syncthreads();

  // Warp 0: claim a tile into slot s (blocking: wait for work; otherwise
  // return at once with go = 2 when nothing is claimable).
  auto claim = [&](int slot, bool blocking) {
    const uint64_t t_acq = globaltimer();
    uint32_t task = 0, phase = 0, tile = 0;
    const int got = acquire<false>(p, cl, task, phase, tile, sh.prof, blocking);
    if (lane == 0) {
      sh.go[slot] = (uint32_t)got;
      sh.task[slot] = task;
      sh.phase[slot] = phase;
      sh.tile[slot] = tile;
    }
    if (got == 1 && lane < (int)(sizeof(TaskBody) / 16)) {
      const uint4 v = ld_cg_v4(reinterpret_cast<const uint4*>(&p.tasks[task].body) + lane);
      reinterpret_cast<uint4*>(&sh.body[slot])[lane] = v;
    }
    __syncwarp();
    if (lane == 0) sh.prof[kProfAcquire] += globaltimer() - t_acq;
  };

  if (warp == 0) claim(0, true);
  __syncthreads();
  int cur = 0;
  while (true) {
    if (sh.go[cur] != 1 || sh.abort) break;
    const int nxt = cur ^ 1;
    const uint64_t t_tile = tid == 0 ? globaltimer() : 0;
    const TaskBody& b = sh.body[cur];
    const uint32_t task = sh.task[cur], tile = sh.tile[cur];
    int bucket = kProfVadd;
    bool early = false;  // warp 0 claims the next tile while this one runs

    if (b.type == kTaskVadd || b.type == kTaskVmul) {
      const int64_t lo = (int64_t)tile * b.vadd_tile;
      const int64_t hi = min(b.n, lo + b.vadd_tile);
      if (warp == 0) {
        claim(nxt, false);
      } else if (b.type == kTaskVadd) {
        vadd_range(reinterpret_cast<const float*>(b.a), reinterpret_cast<const float*>(b.b),
                   reinterpret_cast<float*>(b.c), lo, hi, tid - 32, kThreads - 32);
      } else {
        vmul_range(reinterpret_cast<const float*>(b.a), reinterpret_cast<const float*>(b.b),
                   reinterpret_cast<float*>(b.c), lo, hi, tid - 32, kThreads - 32, b.k);
      }
      early = true;
    } else {
      bucket = kProfGemm;
      const int tm = (int)(tile / b.tiles_n), tn = (int)(tile % b.tiles_n);
      fma_tile(reinterpret_cast<const float*>(b.a), reinterpret_cast<const float*>(b.b),
               reinterpret_cast<float*>(b.c), b.m, (int)b.n, b.k, tm, tn, reinterpret_cast<FmaSmem*>(dyn_smem));
    }
    // need[cur]: the look-ahead claim found nothing, so warp 0 must claim
    // (blocking) after this tile. Written before the barrier and not touched
    // again until two tiles later, so every thread reads the same value (the
    // blocking claim itself rewrites go[nxt] while others may still look).
    if (warp == 0 && lane == 0) {
      if (!early) sh.go[nxt] = 2;
      sh.need[cur] = sh.go[nxt] == 2 ? 1u : 0u;
    }
    // Results written into host memory: visible to the host before the
    // task's completion word.
    if (b.flags & kFlagDirectOut)
      __threadfence_system();
    else
      __threadfence();
    __syncthreads();
    if (sh.abort) {
      if (tid == 0) report_error(p, kStatusTimeout, sh.fail_where, task);
      break;
    }
    if (tid == 0) {
      sh.prof[bucket] += globaltimer() - t_tile;
      sh.prof[kProfTiles] += 1;
      finish_tile(p, task, b.ntiles, b.tag, b.flags);
    }
    if (sh.need[cur]) {
      // Nothing was claimable while the tile ran: wait for work now that its
      // completion is published.
      if (warp == 0) claim(nxt, true);
      __syncthreads();
    }
    cur = nxt;
  }
  __syncthreads();
  if (tid == 0) sched_exit(p, sh.prof);
}

// ---------------------------------------------------------- split3 scheduler
//
// Roles (see gvm_fused.cuh): warp kFzCtlWarp claims tiles and passes them to
// the other warps through a ring of kFzItems items in shared memory; the MMA
// warp and the converter warps each walk the ring in order. GEMM tiles run
// through the fused split3 pipeline (the epilogue of a tile overlaps the
// MMAs of the next); vector-add tiles run on the converter warps. No warp
// waits for another warp's tile to finish except through the pipeline's own
// barriers, so the next tile's claim, staging and MMAs overlap this one's.

constexpr int kFzItems = 4;
constexpr uint32_t kItemExit = 0, kItemNop = 0xffu;  // besides the task types
constexpr int kFinSlots = 16;  // per-item finish counters (items in flight < 16)

// A staged GEMM tile whose accumulator is not drained yet.
struct FzPend {
  uint64_t c;
  int64_t n;
  int32_t m;
  uint32_t tile, tiles_n, task, ntiles, tag, flags, seq;
};

struct FzItem {
  uint32_t kind;  // kItemExit, kItemNop or a task type (kTaskVadd, kTaskSgemm, kTaskVmul)
  uint32_t task;
  uint32_t tile;
  uint32_t tag;
  uint32_t flags;
  uint32_t ntiles;
  uint32_t tiles_n;
  int32_t m;
  int32_t k;
  uint32_t pad;
  int64_t n;
  int64_t vadd_tile;
  uint64_t a, b, c;
  uint64_t tma;  // wide split3: device address of the task's A tensor map, or 0
};

// One thread: ask L2 for a GEMM item's task operands -- A's 128-row block
// of the tile's row (from the tile in column 0 of its row) and all of B
// (from tile (0, 0)) -- so that each task's operands are requested once, in
// pieces of at most 1 MiB, when they are 16-byte aligned, span a multiple
// of 16 bytes and B holds at most 4 MiB. A hint only.
__device__ __forceinline__ void prefetch_task_operands(const FzItem& it) {
  if (it.kind != kTaskSgemm || (it.k & 3) || ((it.a | it.b) & 15)) return;
  const uint32_t tm = it.tile / it.tiles_n, tn = it.tile % it.tiles_n;
  if (tn != 0) return;
  auto pf = [](uint64_t addr, uint64_t bytes) {
    for (uint64_t off = 0; off < bytes; off += (1u << 20)) {
      const uint64_t len = bytes - off < (1u << 20) ? bytes - off : (1u << 20);
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(addr + off), "r"((uint32_t)len) : "memory");
    }
  };
  const int64_t rows = min((int64_t)kTcM, (int64_t)it.m - (int64_t)tm * kTcM);
  if (rows > 0) pf(it.a + (uint64_t)tm * kTcM * (uint64_t)it.k * 4u, (uint64_t)rows * (uint64_t)it.k * 4u);
  const uint64_t b_bytes = (uint64_t)it.k * (uint64_t)it.n * 4u;
  if (tm == 0 && b_bytes <= (4u << 20) && (b_bytes & 15) == 0) pf(it.b, b_bytes);
}

// Shared state of a tensor-core scheduler CTA; Pipe is the tile form's
// pipeline (FzShared: 128 x 256 tiles, WdShared: 256 x 256 tiles).
template <class Pipe>
struct alignas(128) TensorSchedShared {
  Pipe fz;
  uint64_t item_full[kFzItems];   // control -> consumers (1 arrival)
  uint64_t item_empty[kFzItems];  // consumers -> control (converter warps + MMA warp)
  FzItem items[kFzItems];
  uint32_t fin[kFinSlots];        // converter warps done with item (seq % kFinSlots)
  FzPend pend[kFzConvWarps][3];   // per converter warp: GEMM tiles by tile number % 3 (staged, not yet counted)
  uint32_t abort;
  uint32_t fail_where;
  uint64_t prof[kProfSlots];  // kProf* counters; each slot written by one thread only
  uint64_t claim[4];  // Claim state, owned by the control warp
};

// Records a failure seen by this CTA: the CTA flag stops its other warps'
// waits, report_error stops the other CTAs and tells the host.
template <class Sh>
__device__ void cta_fail(const SchedParams& p, Sh& sh, uint32_t where, uint32_t info) {
  sh.fail_where = where;
  sh.abort = 1;
  report_error(p, kStatusTimeout, where, info);
}

// A converter warp has written its share of item `seq` (a vector-add range or
// a drained accumulator). The last of the kFzConvWarps warps completes the
// tile. Lanes fence their own stores before lane 0 counts the warp.
template <class Sh>
__device__ void conv_item_done(const SchedParams& p, Sh& sh, uint32_t seq, uint32_t task, uint32_t ntiles,
                               uint32_t tag, uint32_t flags) {
  // Results written into host memory must be visible to the host before the
  // task's completion word is.
  if (flags & kFlagDirectOut)
    __threadfence_system();
  else
    __threadfence();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) {
    uint32_t* f = &sh.fin[seq % kFinSlots];
    if (atomicAdd(f, 1u) == kFzConvWarps - 1) {
      *f = 0;
      __threadfence();
      finish_tile(p, task, ntiles, tag, flags);
    }
  }
  __syncwarp();
}

// The split3 scheduler CTA for either tile form (kWide: 256 x 256 tiles).
enum : int { kFormFused = 0, kFormWide = 1, kFormTma = 2 };

template <int kForm>
__device__ __forceinline__ void sched_tc_body(const SchedParams& p) {
  constexpr bool kWide = kForm == kFormWide;
  constexpr bool kTma = kForm == kFormTma;
  using Pipe = typename std::conditional<kWide, WdShared,
                                         typename std::conditional<kTma, TmShared, FzShared>::type>::type;
  __shared__ TensorSchedShared<Pipe> sh;
  extern __shared__ uint8_t dyn_smem[];
  uint8_t* stages = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  Claim* cl = reinterpret_cast<Claim*>(sh.claim);
  if (tid == 0) {
    sh.abort = 0;
    sh.fail_where = 0;
    for (int i = 0; i < kProfSlots; ++i) sh.prof[i] = 0;
    for (int i = 0; i < kFinSlots; ++i) sh.fin[i] = 0;
    for (int i = 0; i < kFzItems; ++i) {
      mbar_init(&sh.item_full[i], 1);
      mbar_init(&sh.item_empty[i], kFzConvWarps + (kTma ? 2 : 1));  // converters, MMA (and producer)
    }
    cl->has_resv = 0;
    cl->stall_since = 0;
    cl->hint = ld_relaxed_gpu64(&p.ctrl->first_entry);
    sched_enter(p);
  }
  // initialises the pipeline barriers, fences all inits, allocates TMEM
  if constexpr (kWide)
    wd_init(&sh.fz);
  else if constexpr (kTma)
    tm_init(&sh.fz);
  else
    fz_init(&sh.fz);

  if (warp == kFzCtlWarp) {
    // ---- control: claim tiles into the item ring.
    for (uint32_t seq = 0;; ++seq) {
      const uint32_t slot = seq % kFzItems, ph = (seq / kFzItems) & 1u;
      uint32_t ok = 1;
      if (lane == 0) ok = mbar_wait(&sh.item_empty[slot], ph ^ 1u, p.wait_timeout_ns, &sh.abort) ? 1u : 0u;
      if (!__shfl_sync(0xffffffffu, ok, 0)) {
        if (lane == 0 && !sh.abort) cta_fail(p, sh, kWhereItemRing, seq);
        break;
      }
      const uint64_t t0 = globaltimer();
      uint32_t task = 0, phase = 0, tile = 0;
      // An idle control warp posts a no-op item now and then, so that the
      // other warps' waits for items stay bounded.
      const int got = sh.abort ? 0 : acquire<true>(p, cl, task, phase, tile, sh.prof, true, p.wait_timeout_ns / 4);
      if (lane == 0) {
        FzItem& it = sh.items[slot];
        it.kind = got == 1 ? 0u : (got == 2 ? kItemNop : kItemExit);
        if (got == 1) {
          const TaskBody* b = &p.tasks[task].body;
          it.kind = __ldcg(&b->type);
          it.task = task;
          it.tile = tile;
          it.tag = __ldcg(&b->tag);
          it.flags = __ldcg(&b->flags);
          it.ntiles = __ldcg(&b->ntiles);
          it.tiles_n = __ldcg(&b->tiles_n);
          it.m = __ldcg(&b->m);
          it.k = __ldcg(&b->k);
          it.n = __ldcg(&b->n);
          it.vadd_tile = __ldcg(&b->vadd_tile);
          it.tma = (it.flags & kFlagTmA) ? reinterpret_cast<uint64_t>(&b->tmA) : 0ull;
          it.a = __ldcg(&b->a);
          it.b = __ldcg(&b->b);
          it.c = __ldcg(&b->c);
        }
        sh.prof[kProfAcquire] += globaltimer() - t0;
        mbar_arrive(&sh.item_full[slot]);
        // L2 prefetch, a few tiles ahead of the staging warps: the item two
        // claims back (its slot is rewritten only two claims from now).
        if (p.prefetch && seq >= 2) prefetch_task_operands(sh.items[(seq + 2) % kFzItems]);
      }
      __syncwarp();
      if (got == 0) break;
    }
  } else if (warp == kFzMmaWarp) {
    // ---- MMA issue: GEMM items only; every item is read and released.
    uint32_t it_k = 0, tile_no = 0;
    for (uint32_t seq = 0;; ++seq) {
      const uint32_t slot = seq % kFzItems, ph = (seq / kFzItems) & 1u;
      if (!mbar_wait(&sh.item_full[slot], ph, p.wait_timeout_ns, &sh.abort)) {
        if (lane == 0 && !sh.abort) cta_fail(p, sh, kWhereItemWait, seq);
        break;
      }
      const FzItem& item = sh.items[slot];
      const uint32_t kind = item.kind;
      FzTile t{reinterpret_cast<const float*>(item.a), reinterpret_cast<const float*>(item.b),
               reinterpret_cast<float*>(item.c), item.n, item.m, item.k, 0, 0};
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh.item_empty[slot]);
      if (kind == kItemExit) break;
      if (kind != kTaskSgemm) continue;
      uint32_t ok = 1;
      if (lane == 0) {
        if constexpr (kWide)
          ok = wd_mma(t, stages, &sh.fz, it_k, tile_no, p.wait_timeout_ns, &sh.abort, &sh.fail_where,
                      &sh.prof[kProfMmaWait])
                   ? 1u
                   : 0u;
        else if constexpr (kTma)
          ok = tm_mma(t, stages, &sh.fz, it_k, tile_no, p.wait_timeout_ns, &sh.abort, &sh.fail_where,
                      &sh.prof[kProfMmaWait])
                   ? 1u
                   : 0u;
        else
          ok = fz_mma(t, stages, &sh.fz, it_k, tile_no, p.wait_timeout_ns, &sh.abort, &sh.fail_where,
                      &sh.prof[kProfMmaWait])
                   ? 1u
                   : 0u;
      }
      if (!__shfl_sync(0xffffffffu, ok, 0)) {
        if (lane == 0) report_error(p, kStatusTimeout, sh.fail_where, seq);
        break;
      }
      it_k += (uint32_t)((t.k + kTcBK - 1) / kTcBK);
      ++tile_no;
    }
  } else if (kTma && warp == kTmProducerWarp) {
    // ---- producer (TMA form): every GEMM item's k-steps, in order, get
    // their stage once the MMAs release it, with the tensor copies of A and
    // B when the task has maps.
    if constexpr (kTma) {
      uint32_t it_k = 0, pend[kTcStages] = {0, 0, 0, 0};
      for (uint32_t seq = 0;; ++seq) {
        const uint32_t slot = seq % kFzItems, ph = (seq / kFzItems) & 1u;
        if (!mbar_wait(&sh.item_full[slot], ph, p.wait_timeout_ns, &sh.abort)) {
          if (lane == 0 && !sh.abort) cta_fail(p, sh, kWhereItemWait, seq);
          break;
        }
        const FzItem& item = sh.items[slot];
        const uint32_t kind = item.kind;
        const FzTile t{reinterpret_cast<const float*>(item.a), reinterpret_cast<const float*>(item.b),
                       reinterpret_cast<float*>(item.c), item.n, item.m, item.k,
                       (int)(kind == kTaskSgemm ? item.tile / item.tiles_n : 0),
                       (int)(kind == kTaskSgemm ? item.tile % item.tiles_n : 0)};
        const bool maps = (item.flags & (kFlagTmA | kFlagTmB)) == (kFlagTmA | kFlagTmB);
        const CUtensorMap* tmA = maps ? reinterpret_cast<const CUtensorMap*>(item.tma) : nullptr;
        const CUtensorMap* tmB = maps ? reinterpret_cast<const CUtensorMap*>(item.tma + sizeof(CUtensorMap)) : nullptr;
        const bool b3 = (item.flags & kFlagTmB3) != 0;
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.item_empty[slot]);
        if (kind == kItemExit) break;
        if (kind != kTaskSgemm) continue;
        uint32_t ok = 1;
        if (lane == 0) {
          if (tmA != nullptr) {
            // The maps were written by the ingest's generic stores.
            fence_tensormap_acquire(tmA);
            fence_tensormap_acquire(tmB);
          }
          ok = tm_produce(t, stages, &sh.fz, it_k, tmA, tmB, b3, p.wait_timeout_ns,
                          &sh.abort, &sh.fail_where, pend)
                   ? 1u
                   : 0u;
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) {
          if (lane == 0) report_error(p, kStatusTimeout, sh.fail_where, seq);
          break;
        }
        it_k += (uint32_t)((t.k + kTcBK - 1) / kTcBK);
      }
      if (lane == 0) tm_quiesce(&sh.fz, pend, p.wait_timeout_ns);
      __syncwarp();
    }
  } else if (warp < kFzConvWarps) {
    // ---- converters: stage GEMM tiles; after staging tile T, count tile
    // T-2 as finished (its stores were issued a tile ago, so the fence that
    // orders them before the count hardly waits) and drain tile T-1's
    // accumulator into C. Vector-add tiles, no-op items, the exit and an
    // empty item ring flush both steps first, so that no completion waits
    // for later work.
    uint32_t it_k = 0, tile_no = 0;
    bool has_drain = false, has_done = false;  // tile tile_no-1 to drain; tile done_no to count
    uint32_t done_no = 0;
    uint32_t land_n = 0, land_iss = 0;  // wide form: A landings this warp's group consumed, issued
    // GEMM tile number i of this CTA is kept (by lane 0) in pend[warp][i % 3]
    // until it is counted, out of the registers the staging loop needs.
    auto tile_of = [](const FzItem& item) {
      return FzTile{reinterpret_cast<const float*>(item.a), reinterpret_cast<const float*>(item.b),
                    reinterpret_cast<float*>(item.c), item.n, item.m, item.k,
                    (int)(item.tile / item.tiles_n), (int)(item.tile % item.tiles_n)};
    };
    auto count_done = [&]() {
      if (!has_done) return;
      const FzPend& d = sh.pend[warp][done_no % 3u];
      conv_item_done(p, sh, d.seq, d.task, d.ntiles, d.tag, d.flags);
      has_done = false;
    };
    auto drain = [&]() -> bool {
      if (!has_drain) return true;
      const uint64_t t0 = tid == 0 ? globaltimer() : 0;
      const uint32_t no = tile_no - 1;
      const FzPend& d = sh.pend[warp][no % 3u];
      const FzTile pt{nullptr, nullptr, reinterpret_cast<float*>(d.c), d.n, d.m, 0, (int)(d.tile / d.tiles_n),
                      (int)(d.tile % d.tiles_n)};
      bool drained;
      if constexpr (kWide)
        drained = wd_epilogue(pt, &sh.fz, no, p.wait_timeout_ns, &sh.abort, &sh.fail_where);
      else if constexpr (kTma)
        drained = fz_epilogue(pt, &sh.fz.fz, no, p.wait_timeout_ns, &sh.abort, &sh.fail_where);
      else
        drained = fz_epilogue(pt, &sh.fz, no, p.wait_timeout_ns, &sh.abort, &sh.fail_where);
      if (!drained) return false;
      has_drain = false;
      has_done = true;
      done_no = no;
      if (tid == 0) sh.prof[kProfEpilogue] += globaltimer() - t0;
      return true;
    };
    auto flush = [&]() -> bool {
      count_done();
      if (!drain()) return false;
      count_done();
      return true;
    };
    bool ok = true;
    for (uint32_t seq = 0;; ++seq) {
      const uint32_t slot = seq % kFzItems, ph = (seq / kFzItems) & 1u;
      if ((has_drain || has_done) && !mbar_try_wait(&sh.item_full[slot], ph)) {
        ok = flush();  // nothing queued: finish what is pending before waiting
        if (!ok) break;
      }
      if (!mbar_wait(&sh.item_full[slot], ph, p.wait_timeout_ns, &sh.abort)) {
        if (lane == 0 && !sh.abort) cta_fail(p, sh, kWhereItemWait, seq);
        ok = false;
        break;
      }
      const FzItem& item = sh.items[slot];
      const uint32_t kind = item.kind;
      if (kind == kItemExit || kind == kItemNop) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.item_empty[slot]);
        if (kind == kItemExit) break;
        ok = flush();
        if (!ok) break;
        continue;
      }
      const uint64_t t0 = tid == 0 ? globaltimer() : 0;
      if (kind == kTaskSgemm) {
        const FzTile t = tile_of(item);
        const CUtensorMap* tma = kWide ? reinterpret_cast<const CUtensorMap*>(item.tma) : nullptr;
        const uint32_t item_flags = item.flags;
        __syncwarp();
        if (lane == 0) {
          // The item's sequence number names its finish counter.
          sh.pend[warp][tile_no % 3u] = FzPend{item.c, item.n, item.m, item.tile, item.tiles_n,
                                               item.task, item.ntiles, item.tag, item.flags, seq};
          mbar_arrive(&sh.item_empty[slot]);
        }
        __syncwarp();
        if constexpr (kWide) {
          // One accumulator: drain tile T-1 right after this group's first
          // k-step of T (T's MMAs wait for it), then count T-1.
          // The map was written by the ingest's generic stores: order them
          // before the tensor copies that read it.
          if (tma != nullptr && (warp % kFzGroupWarps) == 0) fence_tensormap_acquire(tma);
          ok = wd_convert(t, stages, &sh.fz, it_k, p.wait_timeout_ns, &sh.abort, &sh.fail_where,
                          tid == 0 ? &sh.prof[kProfStageWait] : nullptr, [&]() -> bool { return drain(); },
                          land_n, land_iss, tma);
          if (ok) ok = drain();  // the group had no k-step of T
          if (ok) count_done();
        } else if constexpr (kTma) {
          const bool landed = (item_flags & (kFlagTmA | kFlagTmB)) == (kFlagTmA | kFlagTmB);
          ok = tm_convert(t, stages, &sh.fz, it_k, landed, p.wait_timeout_ns, &sh.abort, &sh.fail_where,
                          tid == 0 ? &sh.prof[kProfStageWait] : nullptr);
          if (ok) {
            count_done();
            ok = drain();
          }
        } else {
          ok = fz_convert<true>(t, stages, &sh.fz, it_k, p.wait_timeout_ns, &sh.abort, &sh.fail_where,
                                tid == 0 ? &sh.prof[kProfStageWait] : nullptr);
          if (ok) {
            count_done();
            ok = drain();
          }
        }
        it_k += (uint32_t)((t.k + kTcBK - 1) / kTcBK);
        has_drain = true;
        ++tile_no;
        if (tid == 0) sh.prof[kProfGemm] += globaltimer() - t0;
      } else {  // vector add or vector multiply
        const uint32_t task = item.task, ntiles = item.ntiles, tag = item.tag, flags = item.flags;
        const int iters = item.k;
        const int64_t lo = (int64_t)item.tile * item.vadd_tile;
        const int64_t hi = min(item.n, lo + item.vadd_tile);
        const float* a = reinterpret_cast<const float*>(item.a);
        const float* b = reinterpret_cast<const float*>(item.b);
        float* c = reinterpret_cast<float*>(item.c);
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh.item_empty[slot]);
        ok = flush();
        if (ok) {
          if (kind == kTaskVmul) vmul_range(a, b, c, lo, hi, tid, kFzConvThreads, iters);
          else vadd_range(a, b, c, lo, hi, tid, kFzConvThreads);
          conv_item_done(p, sh, seq, task, ntiles, tag, flags);
        }
        if (tid == 0) sh.prof[kProfVadd] += globaltimer() - t0;
      }
      if (tid == 0) sh.prof[kProfTiles] += 1;
      if (!ok) break;
    }
    if (ok && !sh.abort) ok = flush();
    if (!ok && lane == 0) report_error(p, kStatusTimeout, sh.fail_where, 0);
    if constexpr (kWide) wd_land_quiesce(&sh.fz, land_n, land_iss, p.wait_timeout_ns);
  }
  if constexpr (kWide)
    wd_teardown(&sh.fz);
  else if constexpr (kTma)
    fz_teardown(&sh.fz.fz);
  else
    fz_teardown(&sh.fz);
  if (tid == 0) sched_exit(p, sh.prof);
}

__global__ void __launch_bounds__(kFzThreads, 1) sched_fused_kernel(const SchedParams p) {
  sched_tc_body<kFormFused>(p);
}

__global__ void __launch_bounds__(kFzThreads, 1) sched_wide_kernel(const SchedParams p) {
  sched_tc_body<kFormWide>(p);
}

__global__ void __launch_bounds__(kTmThreads, 1) sched_tma_kernel(const SchedParams p) {
  sched_tc_body<kFormTma>(p);
}

static size_t dyn_smem_bytes(int path) {
  if (path == kPathSplit3 || path == kPathSplit3Tma) return (size_t)kTcStages * kTcStageBytes + 1024;
  if (path == kPathSplit3Wide) return (size_t)kWdSmemBytes + 1024;
  return sizeof(FmaSmem) + 1024;
}

static const void* sched_fn(int path) {
  if (path == kPathSplit3) return (const void*)sched_fused_kernel;
  if (path == kPathSplit3Wide) return (const void*)sched_wide_kernel;
  if (path == kPathSplit3Tma) return (const void*)sched_tma_kernel;
  return (const void*)sched_fma_kernel;
}

static int sched_threads(int path) {
  return path == kPathFma ? kThreads : path == kPathSplit3Tma ? kTmThreads : kFzThreads;
}

cudaError_t scheduler_setup(int path, int* blocks_per_sm, size_t* smem_bytes) {
  const size_t smem = dyn_smem_bytes(path);
  const void* fn = sched_fn(path);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, sched_threads(path), smem);
  if (e != cudaSuccess) return e;
  *blocks_per_sm = nb;
  *smem_bytes = smem;
  return cudaSuccess;
}

cudaError_t launch_scheduler(int path, const SchedParams& p, int grid, size_t smem, cudaStream_t stream) {
  if (path == kPathSplit3) {
    sched_fused_kernel<<<grid, kFzThreads, smem, stream>>>(p);
  } else if (path == kPathSplit3Wide) {
    sched_wide_kernel<<<grid, kFzThreads, smem, stream>>>(p);
  } else if (path == kPathSplit3Tma) {
    sched_tma_kernel<<<grid, kTmThreads, smem, stream>>>(p);
  } else {
    sched_fma_kernel<<<grid, kThreads, smem, stream>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace gvm
