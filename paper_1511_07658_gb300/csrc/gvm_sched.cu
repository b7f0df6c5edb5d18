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
//   claim:   entry e at the publication-queue cursor; atomically take the next
//            tile of e's task and phase; advance the cursor when e is used up.
//   ingest:  when nothing is claimable, one CTA (holding a lock) copies ready
//            descriptors from the host rings into the device task table and
//            appends queue entries (split phases of a pass before main phases,
//            so the split3 pre-pass of a task runs well ahead of its GEMM).
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
#include "gvm_runtime.h"

namespace gvm {

struct alignas(128) SchedShared {
  TaskBody body;  // copy of the claimed task's body
  uint32_t go;
  uint32_t task;
  uint32_t phase;
  uint32_t tile;
  uint32_t abort;
  uint32_t fail_where;
  uint32_t pad[2];
  uint64_t prof[8];  // this CTA's phase counters (kProf*), written by thread 0 only
  TcShared tc;
};

constexpr uint32_t kMaxQuantum = 8;
constexpr uint64_t kLookahead = 16;  // ingest ahead when this few queue entries remain
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
// device table and the publication queue. All lanes call.
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
  const uint64_t pub0 = ld_relaxed_gpu64(&p.ctrl->published);
  const uint64_t cur = ld_relaxed_gpu64(&p.ctrl->cursor);
  const uint32_t rr = ld_relaxed_gpu(&p.ctrl->rr);
  const uint64_t now = globaltimer();
  uint64_t pub = pub0;
  uint32_t pending = 0;
  bool bad = false;

  for (uint32_t g = 0; g < p.ranks; g += 32) {
    const uint32_t used = (uint32_t)(pub - cur);
    const uint32_t space = used < p.qcap ? p.qcap - used : 0u;
    uint32_t quantum = min(p.quantum, kMaxQuantum);
    // Each task takes at most two queue entries; keep this pass within the free space.
    const uint32_t lanes = min(32u, p.ranks - g);
    if (2u * lanes * quantum > space) quantum = space / (2u * lanes);

    uint32_t r = 0, t = 0, take = 0, avail = 0;
    const bool valid = (g + lane) < p.ranks;
    if (valid) {
      r = (rr + g + lane) % p.ranks;
      const uint32_t h = ld_acquire_sys(&p.host_heads[r].head);
      t = ld_relaxed_gpu(&p.tail[r]);
      avail = h - t;
      const uint32_t lim = min(avail, quantum);
      for (; take < lim; ++take) {
        const uint32_t s = t + take;
        const uint32_t idx = r * p.depth + (s & (p.depth - 1));
        const uint32_t flags = ld_volatile_u32(&p.host_desc[idx].flags);
        if ((flags & kFlagNeedsReady) && ld_acquire_gpu(&p.ready[idx]) != s + 1u) break;
      }
    }

    uint32_t tidx[kMaxQuantum];
    uint32_t kinds = 0;  // bit 2i: has split entry, bit 2i+1: has main entry
    uint32_t nsplit_e = 0, nmain_e = 0;
    for (uint32_t i = 0; i < take; ++i) {
      const uint32_t s = t + i;
      const uint32_t idx = r * p.depth + (s & (p.depth - 1));
      tidx[i] = idx;
      DevTask* dt = &p.tasks[idx];
      atomicExch(&dt->claimed[0], kClaimLocked);
      atomicExch(&dt->claimed[1], kClaimLocked);
      const uint4* src = reinterpret_cast<const uint4*>(&p.host_desc[idx]);
      uint4* dst = reinterpret_cast<uint4*>(&dt->body);
#pragma unroll
      for (int blk = 0; blk < 3; ++blk) {
        uint4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = ld_volatile_v4(src + blk * 8 + j);
#pragma unroll
        for (int j = 0; j < 8; ++j) st_cg_v4(dst + blk * 8 + j, v[j]);
      }
      const TaskBody* hb = &p.host_desc[idx];
      const uint32_t tag = ld_volatile_u32(&hb->tag);
      const uint32_t ntiles = ld_volatile_u32(&hb->ntiles);
      const uint32_t nsplit = ld_volatile_u32(&hb->nsplit);
      const uint32_t flags = ld_volatile_u32(&hb->flags);
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
      if (nsplit > 0) {
        kinds |= 1u << (2 * i);
        ++nsplit_e;
      }
      if (ntiles > nsplit) {
        kinds |= 1u << (2 * i + 1);
        ++nmain_e;
      }
    }
    const uint32_t incl_s = warp_incl_scan(nsplit_e);
    const uint32_t incl_m = warp_incl_scan(nmain_e);
    const uint32_t tot_s = __shfl_sync(0xffffffffu, incl_s, 31);
    const uint32_t tot_m = __shfl_sync(0xffffffffu, incl_m, 31);
    uint64_t ps = pub + incl_s - nsplit_e;
    uint64_t pm = pub + tot_s + incl_m - nmain_e;
    for (uint32_t i = 0; i < take; ++i) {
      if (kinds & (1u << (2 * i))) {
        PubEntry e{tidx[i], kPhaseSplit};
        p.pubq[ps++ & (p.qcap - 1)] = e;
      }
      if (kinds & (1u << (2 * i + 1))) {
        PubEntry e{tidx[i], kPhaseMain};
        p.pubq[pm++ & (p.qcap - 1)] = e;
      }
    }
    __threadfence();
    fence_tensormap_release();
    for (uint32_t i = 0; i < take; ++i) {
      if (kinds & (3u << (2 * i))) {
        atomicExch(&p.tasks[tidx[i]].claimed[0], 0u);
        atomicExch(&p.tasks[tidx[i]].claimed[1], 0u);
      }
    }
    if (valid && take > 0) *reinterpret_cast<volatile uint32_t*>(&p.tail[r]) = t + take;
    pending += avail - take;
    pub += tot_s + tot_m;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) pending += __shfl_xor_sync(0xffffffffu, pending, d);
  const uint32_t any_bad = __any_sync(0xffffffffu, bad);
  __threadfence();
  if (lane == 0) {
    if (pending == 0 && pub == pub0)
      *reinterpret_cast<volatile uint64_t*>(&p.ctrl->quiet_until) = now + kQuietNs;
    if (pub != pub0) st_release_gpu64(&p.ctrl->published, pub);
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

// Warp 0: find the next tile to run. Returns 1 with (task, phase, tile) set,
// or 0 when the kernel should exit. Every decision is taken on values lane 0
// read and broadcast, so the warp never diverges across the shuffles.
__device__ int acquire(const SchedParams& p, uint32_t& task, uint32_t& phase, uint32_t& tile,
                       uint64_t& idle_since, uint64_t* prof) {
  const int lane = threadIdx.x & 31;
  uint64_t stall_since = 0;
  while (true) {
    uint32_t abort = 0, drained = 0;
    uint64_t cur = 0, pub = 0, now = 0, quiet = 0;
    if (lane == 0) {
      abort = ld_relaxed_gpu(&p.ctrl->abort);
      drained = ld_relaxed_gpu(&p.ctrl->drained);
      cur = ld_relaxed_gpu64(&p.ctrl->cursor);
      pub = ld_acquire_gpu64(&p.ctrl->published);
      quiet = ld_relaxed_gpu64(&p.ctrl->quiet_until);
      now = globaltimer();
    }
    if (bcast(abort)) return 0;
    drained = bcast(drained);
    cur = bcast64(cur);
    pub = bcast64(pub);
    now = bcast64(now);
    quiet = bcast64(quiet);
    if (cur < pub) {
      // Keep the queue ahead of the CTAs, unless a recent pass found the rings empty.
      if (pub - cur <= kLookahead && now >= quiet) (void)ingest(p, prof);
      uint32_t x = 0, etask = 0, ephase = 0, cnt = 0;
      if (lane == 0) {
        const uint64_t raw = ld_relaxed_gpu64(reinterpret_cast<const uint64_t*>(&p.pubq[cur & (p.qcap - 1)]));
        etask = (uint32_t)raw;
        ephase = (uint32_t)(raw >> 32) & 1u;
        x = atomicAdd(&p.tasks[etask].claimed[ephase], 1u);
        __threadfence();
        const TaskBody* b = &p.tasks[etask].body;
        const uint32_t ntiles = ld_relaxed_gpu(&b->ntiles);
        const uint32_t nsplit = ld_relaxed_gpu(&b->nsplit);
        cnt = (ephase == kPhaseSplit) ? nsplit : ntiles - nsplit;
        if (x >= cnt)
          atomicMax(reinterpret_cast<unsigned long long*>(&p.ctrl->cursor), (unsigned long long)(cur + 1));
      }
      x = bcast(x);
      cnt = bcast(cnt);
      if (x < cnt) {
        task = bcast(etask);
        phase = bcast(ephase);
        tile = x;
        idle_since = 0;
        return 1;
      }
      continue;
    }
    if (p.drain && drained) return 0;
    const IngestOut r = ingest(p, prof);
    if (r.published) {
      stall_since = 0;
      idle_since = 0;
      continue;
    }
    if (!r.locked_out) {
      if (r.pending == 0) {
        stall_since = 0;
        if (p.drain) {
          if (lane == 0) atomicExch(&p.ctrl->drained, 1u);
          __syncwarp();
          return 0;
        }
        uint32_t stop = 0;
        if (lane == 0) stop = ld_acquire_sys(&p.host_shared->stop);
        if (bcast(stop)) return 0;
      } else {
        if (stall_since == 0) stall_since = now;
        else if (now - stall_since > p.wait_timeout_ns) {
          if (lane == 0) report_error(p, kStatusTimeout, kWhereReadyWait, r.pending);
          __syncwarp();
          return 0;
        }
      }
    }
    __nanosleep(r.locked_out ? 200u : (uint32_t)p.idle_poll_ns);
  }
}

template <int PATH>
__global__ void __launch_bounds__(kThreads, PATH == kPathFma ? 2 : 1) sched_kernel(const SchedParams p) {
  __shared__ SchedShared sh;
  extern __shared__ uint8_t dyn_smem[];
  uint8_t* big = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    sh.abort = 0;
    sh.fail_where = 0;
    for (int i = 0; i < 8; ++i) sh.prof[i] = 0;
    const unsigned long long t0 = globaltimer();
    unsigned long long* ts = reinterpret_cast<unsigned long long*>(&p.ctrl->t_start);
    if (atomicCAS(ts, 0ull, t0) != 0ull) atomicMin(ts, t0);
  }
  uint32_t it = 0, tile_no = 0;
  if constexpr (PATH == kPathSplit3) {
    tc_init(&sh.tc);
  } else {
    __syncthreads();
  }
  uint64_t idle_since = 0;

  while (true) {
    if (warp == 0) {
      const uint64_t t_acq = globaltimer();
      uint32_t task = 0, phase = 0, tile = 0;
      const int got = acquire(p, task, phase, tile, idle_since, sh.prof);
      if (lane == 0) {
        sh.go = (uint32_t)got;
        sh.task = task;
        sh.phase = phase;
        sh.tile = tile;
      }
      if (got && lane < (int)(sizeof(TaskBody) / 16)) {
        const uint4 v = ld_cg_v4(reinterpret_cast<const uint4*>(&p.tasks[task].body) + lane);
        reinterpret_cast<uint4*>(&sh.body)[lane] = v;
      }
      if (lane == 0) sh.prof[kProfAcquire] += globaltimer() - t_acq;
    }
    __syncthreads();
    if (!sh.go || sh.abort) break;
    const uint64_t t_tile = tid == 0 ? globaltimer() : 0;
    const TaskBody& b = sh.body;
    const uint32_t task = sh.task, phase = sh.phase, tile = sh.tile;
    int bucket = kProfVadd;

    if (b.type == kTaskVadd) {
      const int64_t lo = (int64_t)tile * b.vadd_tile;
      const int64_t hi = min(b.n, lo + b.vadd_tile);
      vadd_range(reinterpret_cast<const float*>(b.a), reinterpret_cast<const float*>(b.b),
                 reinterpret_cast<float*>(b.c), lo, hi);
    } else {
      const float* A = reinterpret_cast<const float*>(b.a);
      const float* B = reinterpret_cast<const float*>(b.b);
      float* C = reinterpret_cast<float*>(b.c);
      if constexpr (PATH == kPathFma) {
        bucket = kProfGemm;
        const int tm = (int)(tile / b.tiles_n), tn = (int)(tile % b.tiles_n);
        fma_tile(A, B, C, b.m, (int)b.n, b.k, tm, tn, reinterpret_cast<FmaSmem*>(big));
      } else {
        if (phase == kPhaseSplit) {
          bucket = kProfSplit;
          const uint32_t tiles_a = (uint32_t)((b.m + kSplitRows - 1) / kSplitRows);
          if (tile < tiles_a) {
            split_a_tile(A, reinterpret_cast<__nv_bfloat16*>(b.scratch), b.m, b.k, (int)b.kp,
                         (int)(tile * kSplitRows), kSplitRows);
          } else {
            split_b_tile(B, reinterpret_cast<__nv_bfloat16*>(b.scratch_b), b.n, b.k, (int)b.kp,
                         (int64_t)(tile - tiles_a) * kSplitRows, kSplitRows);
          }
          fence_proxy_async_global();
        } else {
          bucket = kProfGemm;
          const int tm = (int)(tile / b.tiles_n), tn = (int)(tile % b.tiles_n);
          const DevTask* dt = &p.tasks[task];
          tc_tile(&dt->body.tmA, &dt->body.tmB, C, b.m, b.n, b.k, tm, tn, big, &sh.tc, it, tile_no,
                  p.wait_timeout_ns, b.nsplit ? &dt->split_done : nullptr, b.nsplit, &sh.abort,
                  &sh.fail_where, true, &sh.prof[kProfSplitWait]);
        }
      }
    }
    __threadfence();
    __syncthreads();
    if (sh.abort) {
      if (tid == 0) report_error(p, kStatusTimeout, sh.fail_where, task);
      break;
    }
    if (tid == 0) {
      sh.prof[bucket] += globaltimer() - t_tile;
      sh.prof[kProfTiles] += 1;
      DevTask* dt = &p.tasks[task];
      if (phase == kPhaseSplit) atomicAdd(&dt->split_done, 1u);
      const uint32_t d = atomicAdd(&dt->tiles_done, 1u);
      if (d + 1 == b.ntiles) {
        __threadfence();
        const uint64_t t_in = *reinterpret_cast<volatile uint64_t*>(&dt->t_ingest);
        complete_task(p, task, b.tag, b.flags, t_in);
      }
    }
  }

  if constexpr (PATH == kPathSplit3) {
    tc_teardown(&sh.tc);
  }
  if (tid == 0) {
    for (int i = 0; i < 8; ++i)
      atomicAdd(reinterpret_cast<unsigned long long*>(&p.ctrl->prof[i]), (unsigned long long)sh.prof[i]);
    __threadfence();
    const uint32_t n = atomicAdd(&p.ctrl->exit_count, 1u);
    if (n + 1 == gridDim.x) {
      // Every CTA has left: publish this launch's timeline and phase
      // counters, then reset the per-launch words for the next launch.
      HostShared* hs = p.host_shared;
      st_relaxed_sys64(&hs->k_start, atomicExch(reinterpret_cast<unsigned long long*>(&p.ctrl->t_start), 0ull));
      st_relaxed_sys64(&hs->k_last_done,
                       atomicExch(reinterpret_cast<unsigned long long*>(&p.ctrl->t_last_done), 0ull));
      for (int i = 0; i < 8; ++i)
        st_relaxed_sys64(&hs->k_prof[i], atomicExch(reinterpret_cast<unsigned long long*>(&p.ctrl->prof[i]), 0ull));
      st_relaxed_sys64(&hs->k_exit, globaltimer());
      atomicExch(&p.ctrl->exit_count, 0u);
      atomicExch(&p.ctrl->drained, 0u);
      atomicExch(&p.ctrl->ingest_lock, 0u);
      __threadfence_system();
      st_release_sys(&p.host_shared->exit_gen, p.launch_gen);
    }
  }
}

static size_t dyn_smem_bytes(int path) {
  return (path == kPathSplit3 ? (size_t)kTcStages * kTcStageBytes : sizeof(FmaSmem)) + 1024;
}

cudaError_t scheduler_setup(int path, int* blocks_per_sm, size_t* smem_bytes) {
  const size_t smem = dyn_smem_bytes(path);
  const void* fn = path == kPathSplit3 ? (const void*)sched_kernel<kPathSplit3> : (const void*)sched_kernel<kPathFma>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, smem);
  if (e != cudaSuccess) return e;
  *blocks_per_sm = nb;
  *smem_bytes = smem;
  return cudaSuccess;
}

cudaError_t launch_scheduler(int path, const SchedParams& p, int grid, size_t smem, cudaStream_t stream) {
  if (path == kPathSplit3) {
    sched_kernel<kPathSplit3><<<grid, kThreads, smem, stream>>>(p);
  } else {
    sched_kernel<kPathFma><<<grid, kThreads, smem, stream>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace gvm
