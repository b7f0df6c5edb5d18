// Split3 SGEMM on CTA pairs: the fused staging of gvm_fused.cuh with
// two-SM tensor-core MMAs (tcgen05 cta_group::2).
//
// A cluster of two CTAs on neighbouring SMs computes one 256 x 256 tile of C.
// Each CTA stages its own 128 rows of A and its own 128 columns of B (split
// into bf16 hi and lo planes as in gvm_fused.cuh); one thread of the even
// CTA (the leader) issues 256 x 256 x 16 MMAs that read A and B from both
// CTAs' shared memory and accumulate each CTA's 128 rows in its own TMEM.
// Per SM and per k-step a CTA therefore loads, splits and stores 8192
// operand values instead of 12288 for the same tensor work, so the same
// bytes in flight per SM cover 1.5 times the tensor work.
//
// Roles are those of gvm_fused.cuh (warps 0-7 stage and drain, warp 8 MMA,
// warp 9 claims), except that all 8 staging warps take every k-step; in the
// peer CTA warp 8 relays the peer's arrivals to the leader. Barriers:
//   full[s]      leader only: its 8 staging warps arrive, and the peer's
//                relay once for the peer's 8; then the leader issues MMAs;
//   empty[s]     both CTAs: the leader's commit arrives in both (multicast);
//   acc_full[b]  both CTAs: the leader's commit after a tile's last k-step;
//   acc_empty[b] leader only: its 8 staging warps and the relay (for the
//                peer's 8) arrive once accumulator b is drained;
//   pfull[s], pdrained[b]  peer only: its staging warps, for the relay.
//
// Stage layout (kPrStageBytes = 32 KB): A hi, A lo [128 rows][32 k] K-major;
// B hi, B lo [32 k][128 n] MN-major (4 atoms of 32 columns, 512 B apart;
// 8-row k groups 2048 B apart); the 64-byte swizzle of gvm_fused.cuh. The
// stage buffers sit at the same shared-memory offsets in both CTAs (the
// MMA's descriptors name offsets the hardware reads in each CTA).
#pragma once

#include "gvm_fused.cuh"

namespace gvm {

constexpr int kPrM = 2 * kTcM;  // rows of a pair tile
constexpr int kPrN = kTcN;      // columns of a pair tile (each CTA stages half)
constexpr int kPrMaxStages = 6;
constexpr int kPrDefaultStages = 4;  // 128 KB of stages: the rest of the SM's 256 KB stays L1
constexpr uint32_t kPrAOff = 0;
constexpr uint32_t kPrAlOff = kTcM * kTcBK * 2;
constexpr uint32_t kPrBOff = 2 * kTcM * kTcBK * 2;
constexpr uint32_t kPrBlOff = kPrBOff + (kPrN / 2) * kTcBK * 2;
constexpr uint32_t kPrStageBytes = kPrBlOff + (kPrN / 2) * kTcBK * 2;
static_assert(kPrStageBytes == 32768, "pair stage layout");
constexpr uint32_t kPrBAtomN = 512;   // 32 columns x 8 k rows x 2 B
constexpr uint32_t kPrBAtomK = 2048;  // 4 column atoms
// Instruction descriptor: bf16 x bf16 -> fp32, A K-major, B MN-major, M 256, N 256.
constexpr uint32_t kPrIdesc = idesc_bf16_f32(kPrM, kPrN) | (1u << 16);

struct PrShared {
  uint64_t full[kPrMaxStages];   // leader: its 8 staging warps + the relay's 8
  uint64_t empty[kPrMaxStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];         // leader: its 8 staging warps + the relay's 8
  uint64_t pfull[kPrMaxStages];  // peer: its 8 staging warps (for the relay)
  uint64_t pdrained[2];          // peer: its 8 staging warps (for the relay)
  uint32_t tmem_base;
  uint32_t cta;      // rank of this CTA in its pair (0 = leader)
  uint32_t nstages;  // pipeline stages in use (<= kPrMaxStages)
  uint32_t pad;
};

// ---------------------------------------------------------------- cluster PTX

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Shared::cluster address of the same shared-memory location in CTA `rank`.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait with cluster-scope acquire (arrivals from the other CTA).
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, uint64_t timeout_ns,
                                                  volatile uint32_t* cta_abort) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t deadline = globaltimer() + timeout_ns;
  while (true) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if (*cta_abort) return false;
    if (globaltimer() > deadline) return false;
  }
}
// Whole-cluster barrier; every thread of both CTAs must reach it.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void st_cluster_v4(uint32_t cluster_addr, uint4 v) {
  asm volatile("st.shared::cluster.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(cluster_addr), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}
__device__ __forceinline__ void umma_bf16_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                               uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrives on `bar` (same offset) in both CTAs once the MMAs issued so far are done.
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"((uint16_t)3)
      : "memory");
}
__device__ __forceinline__ uint64_t sdesc_mn64b_pair(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(kPrBAtomN >> 4) << 16;
  d |= (uint64_t)(kPrBAtomK >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Both CTAs: barriers, then (warp 8 of each CTA) the pair's TMEM, then a
// cluster barrier so that no CTA arrives on the other's barriers before they
// exist.
__device__ __forceinline__ void pr_init(PrShared* ps, uint32_t nstages) {
  if (threadIdx.x == 0) {
    ps->cta = cluster_ctarank();
    ps->nstages = nstages;
    for (int s = 0; s < kPrMaxStages; ++s) {
      mbar_init(&ps->full[s], 2 * kFzConvWarps);
      mbar_init(&ps->empty[s], 1);
      mbar_init(&ps->pfull[s], kFzConvWarps);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ps->acc_full[b], 1);
      mbar_init(&ps->acc_empty[b], 2 * kFzConvWarps);
      mbar_init(&ps->pdrained[b], kFzConvWarps);
    }
    mbar_fence_init();
  }
  if ((threadIdx.x >> 5) == kFzMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&ps->tmem_base)),
                 "r"(kFzTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
}

// Both CTAs, every thread: after all of the pair's MMAs have completed
// (every staging warp drained its accumulators), free the TMEM.
__device__ __forceinline__ void pr_teardown(PrShared* ps) {
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  if ((threadIdx.x >> 5) == kFzMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(ps->tmem_base), "r"(kFzTmemCols)
                 : "memory");
}

// ---------------------------------------------------------------- staging

// All 8 staging warps take part in every k-step; thread (w, lane) of warp w
// stages, of its CTA's half of pair tile (tm, tn), k-step kb:
//   A item j (j = 0, 1): atom a = w + 8 j, row 8 a + (lane >> 2) of the CTA's
//                        128 rows, 8 values from k = 32 kb + 8 (lane & 3);
//   B item j (j = 0, 1): atom a = w + 8 j, k = 32 kb + 8 (a >> 2) + (lane >> 2),
//                        8 values from column 32 (a & 3) + 8 (lane & 3) of the
//                        CTA's 128 columns.
// Each store instruction of a warp fills one 512-byte swizzle atom.
__device__ __forceinline__ void pr_load_a(const FzTile& t, int row0, int kb, int w, int lane, int j, int avec,
                                          float (&v)[8]) {
  const int r = row0 + 8 * (w + 8 * j) + (lane >> 2);
  const int kk = kb * kTcBK + 8 * (lane & 3);
  const float* src = t.A + (int64_t)r * t.k + kk;
  if (r < t.m && avec == 2 && kk + 8 <= t.k) {
    ld_cg_v8(src, v);
  } else if (r < t.m && avec && kk + 8 <= t.k) {
    const float4 x0 = __ldcg(reinterpret_cast<const float4*>(src));
    const float4 x1 = __ldcg(reinterpret_cast<const float4*>(src + 4));
    v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
    v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (r < t.m && kk + e < t.k) ? __ldcg(src + e) : 0.f;
  }
}
__device__ __forceinline__ void pr_load_b(const FzTile& t, int64_t col0, int kb, int w, int lane, int j, int bvec,
                                          float (&v)[8]) {
  const int a = w + 8 * j;
  const int kk = kb * kTcBK + 8 * (a >> 2) + (lane >> 2);
  const int64_t c = col0 + 32 * (a & 3) + 8 * (lane & 3);
  const float* src = t.B + (int64_t)kk * t.n + c;
  if (kk < t.k && bvec == 2 && c + 8 <= t.n) {
    ld_cg_v8(src, v);
  } else if (kk < t.k && bvec && c + 8 <= t.n) {
    const float4 x0 = __ldcg(reinterpret_cast<const float4*>(src));
    const float4 x1 = __ldcg(reinterpret_cast<const float4*>(src + 4));
    v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
    v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (kk < t.k && c + e < t.n) ? __ldcg(src + e) : 0.f;
  }
}

// Register prefetch depth of the pair staging warps on interior tiles
// (k-steps): at this depth a thread holds as many bytes in flight (96
// floats) as in the single-CTA form, for two thirds of the bytes per k-step.
// Ragged tiles, whose loads check bounds, keep two k-steps in flight.
constexpr int kPrDepth = 2;

// Staging warps of both CTAs: every k-step of pair tile (t.tm, t.tn), this
// CTA's half of it. `it` counts k-steps before this tile (same in every
// role of both CTAs). A k-step is announced on `arrive_to` (the leader's
// full[s] in the leader, the relay's pfull[s] in the peer). kFast: the
// CTA's half lies inside A, B and C, k is a multiple of kTcBK and rows are
// 32-byte aligned; each item is then one 32-byte load at a fixed offset from
// two per-thread bases.
template <bool kFast, int kDepth>
__device__ __forceinline__ bool pr_convert_loop(const FzTile& t, uint32_t base, PrShared* ps, uint64_t* arrive_to,
                                                uint32_t it, int avec, int bvec, uint64_t timeout_ns,
                                                volatile uint32_t* cta_abort, uint32_t* fail_where,
                                                uint64_t* wait_acc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t cta = ps->cta, ns = ps->nstages;
  const int nkb = (t.k + kTcBK - 1) / kTcBK;
  const int row0 = t.tm * kPrM + (int)cta * kTcM;
  const int64_t col0 = (int64_t)t.tn * kPrN + (int64_t)cta * (kPrN / 2);
  // Fast path: items j = 0, 1 of A are 64 rows apart, of B 16 rows apart;
  // a k-step moves A by kTcBK columns and B by kTcBK rows.
  const float* pa0 = t.A + (int64_t)(row0 + 8 * warp + (lane >> 2)) * t.k + 8 * (lane & 3);
  const float* pb0 = t.B + (int64_t)(8 * (warp >> 2) + (lane >> 2)) * t.n + col0 + 32 * (warp & 3) + 8 * (lane & 3);
  const float* pa1 = pa0 + 64 * (int64_t)t.k;
  const float* pb1 = pb0 + 16 * t.n;
  const uint32_t b_step = (uint32_t)kTcBK * (uint32_t)t.n;
  auto load_a = [&](int kb, int j, float (&v)[8]) {
    if (kFast) ld_cg_v8((j ? pa1 : pa0) + (uint32_t)kb * (uint32_t)kTcBK, v);
    else pr_load_a(t, row0, kb, warp, lane, j, avec, v);
  };
  auto load_b = [&](int kb, int j, float (&v)[8]) {
    if (kFast) ld_cg_v8((j ? pb1 : pb0) + (uint64_t)(uint32_t)kb * b_step, v);
    else pr_load_b(t, col0, kb, warp, lane, j, bvec, v);
  };
  float va[kDepth][2][8], vb[kDepth][2][8];
#pragma unroll
  for (int d = 0; d < kDepth; ++d) {
    if (d < nkb) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        load_a(d, j, va[d][j]);
        load_b(d, j, vb[d][j]);
      }
    }
  }
  const uint32_t sw = swz64((uint32_t)(lane >> 2), (uint32_t)(lane & 3));
  // k-steps in blocks of kDepth, so that the register buffers stay
  // statically indexed.
  for (int kb0 = 0; kb0 < nkb; kb0 += kDepth) {
#pragma unroll
    for (int d = 0; d < kDepth; ++d) {
      const int kb = kb0 + d;
      if (kb < nkb) {
        const uint32_t q = it + (uint32_t)kb, s = q % ns, ph = (q / ns) & 1u;
        uint64_t t0 = 0;
        if (wait_acc != nullptr && warp == 0 && lane == 0) t0 = globaltimer();
        if (!mbar_wait(&ps->empty[s], ph ^ 1u, timeout_ns, cta_abort)) {
          if (lane == 0) {
            *fail_where = kWhereEmptyBarrier;
            *cta_abort = 1;
          }
          return false;
        }
        if (t0) *wait_acc += globaltimer() - t0;
        const uint32_t st = base + s * kPrStageBytes;
        const bool more = kb + kDepth < nkb;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const uint32_t a = (uint32_t)(warp + 8 * j);
          uint4 hi, lo;
          split8_x2(va[d][j], hi, lo);
          st_shared_v4(st + kPrAOff + a * 512u + sw, hi);
          st_shared_v4(st + kPrAlOff + a * 512u + sw, lo);
          if (more) load_a(kb + kDepth, j, va[d][j]);
          const uint32_t boff = (a >> 2) * kPrBAtomK + (a & 3u) * kPrBAtomN + sw;
          split8_x2(vb[d][j], hi, lo);
          st_shared_v4(st + kPrBOff + boff, hi);
          st_shared_v4(st + kPrBlOff + boff, lo);
          if (more) load_b(kb + kDepth, j, vb[d][j]);
        }
        fence_proxy_async_shared();
        __syncwarp();
        if (lane == 0) mbar_arrive(&arrive_to[s]);
      }
    }
  }
  return true;
}

__device__ __forceinline__ bool pr_convert(const FzTile& t, uint8_t* stages, PrShared* ps, uint64_t* arrive_to,
                                           uint32_t it, uint64_t timeout_ns, volatile uint32_t* cta_abort,
                                           uint32_t* fail_where, uint64_t* wait_acc) {
  const int avec = ((t.k & 7) == 0 && (reinterpret_cast<uintptr_t>(t.A) & 31) == 0)   ? 2
                   : ((t.k & 3) == 0 && (reinterpret_cast<uintptr_t>(t.A) & 15) == 0) ? 1
                                                                                      : 0;
  const int bvec = ((t.n & 7) == 0 && (reinterpret_cast<uintptr_t>(t.B) & 31) == 0)   ? 2
                   : ((t.n & 3) == 0 && (reinterpret_cast<uintptr_t>(t.B) & 15) == 0) ? 1
                                                                                      : 0;
  const int row_end = t.tm * kPrM + ((int)ps->cta + 1) * kTcM;
  const int64_t col_end = (int64_t)t.tn * kPrN + (int64_t)(ps->cta + 1) * (kPrN / 2);
  const bool fast = avec == 2 && bvec == 2 && (t.k % kTcBK) == 0 && row_end <= t.m && col_end <= t.n;
  const uint32_t base = smem_u32(stages);
  return fast ? pr_convert_loop<true, kPrDepth>(t, base, ps, arrive_to, it, avec, bvec, timeout_ns, cta_abort,
                                                fail_where, wait_acc)
              : pr_convert_loop<false, 2>(t, base, ps, arrive_to, it, avec, bvec, timeout_ns, cta_abort, fail_where,
                                          wait_acc);
}

// Peer CTA, one lane of warp 8: forwards the peer's local "stage filled" and
// "accumulator drained" arrivals to the leader, one cluster-scope release
// per event. Issued from the staging warps themselves, each release would
// wait for that warp's loads in flight (a cluster-scope release orders all
// of a thread's prior memory operations).
// `bar` names a barrier by its offset in this CTA; the arrival goes to the
// barrier at that offset in the leader.
__device__ __forceinline__ void pr_relay_forward(uint64_t* bar, uint32_t count) {
  fence_proxy_async_shared();
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(mapa_shared(smem_u32(bar), 0)),
               "r"(count)
               : "memory");
}

// The relay over the same tile sequence as the staging warps: k-step
// arrivals of tile number tile_no, then the drain of tile_no - 1.
__device__ __forceinline__ bool pr_relay_tile(PrShared* ps, uint32_t it, int nkb, uint32_t tile_no,
                                              uint64_t timeout_ns, volatile uint32_t* cta_abort,
                                              uint32_t* fail_where) {
  const uint32_t ns = ps->nstages;
  for (int kb = 0; kb < nkb; ++kb) {
    const uint32_t q = it + (uint32_t)kb, s = q % ns, ph = (q / ns) & 1u;
    if (!mbar_wait(&ps->pfull[s], ph, timeout_ns, cta_abort)) {
      *fail_where = kWhereFullBarrier;
      *cta_abort = 1;
      return false;
    }
    pr_relay_forward(&ps->full[s], kFzConvWarps);
  }
  return true;
}
__device__ __forceinline__ bool pr_relay_drain(PrShared* ps, uint32_t tile_no, uint64_t timeout_ns,
                                               volatile uint32_t* cta_abort, uint32_t* fail_where) {
  const uint32_t b = tile_no & 1u;
  if (!mbar_wait(&ps->pdrained[b], (tile_no >> 1) & 1u, timeout_ns, cta_abort)) {
    *fail_where = kWhereAccumBarrier;
    *cta_abort = 1;
    return false;
  }
  pr_relay_forward(&ps->acc_empty[b], kFzConvWarps);
  return true;
}

// Staging warps of both CTAs: drain this CTA's half (128 rows) of
// accumulator (tile_no & 1) into C, then tell the leader.
__device__ __forceinline__ bool pr_epilogue(const FzTile& t, PrShared* ps, uint32_t tile_no, uint64_t timeout_ns,
                                            volatile uint32_t* cta_abort, uint32_t* fail_where) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t b = tile_no & 1u;
  if (!mbar_wait(&ps->acc_full[b], (tile_no >> 1) & 1u, timeout_ns, cta_abort)) {
    if (lane == 0) {
      *fail_where = kWhereAccumBarrier;
      *cta_abort = 1;
    }
    return false;
  }
  tc_fence_after();
  const int q = warp & 3, cq = warp >> 2;
  const int row = t.tm * kPrM + (int)ps->cta * kTcM + q * 32 + lane;
  const uintptr_t ca = reinterpret_cast<uintptr_t>(t.C);
  const int vec = ((t.n & 7) == 0 && (ca & 31) == 0) ? 2 : ((t.n & 3) == 0 && (ca & 15) == 0) ? 1 : 0;
#pragma unroll 1
  for (int ch = 0; ch < 4; ++ch) {
    const int chunk = cq * 4 + ch;
    uint32_t r[32];
    tmem_ld_32x32b_x32(ps->tmem_base + b * kTcN + ((uint32_t)(q * 32) << 16) + (uint32_t)(chunk * 32), r);
    tmem_ld_wait();
    const int64_t c0 = (int64_t)t.tn * kPrN + chunk * 32;
    if (row < t.m && c0 < t.n) {
      float* dst = t.C + (int64_t)row * t.n + c0;
      if (vec == 2 && c0 + 32 <= t.n) {
#pragma unroll
        for (int j = 0; j < 4; ++j) st_v8(dst + 8 * j, r + 8 * j);
      } else if (vec == 1 && c0 + 32 <= t.n) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          reinterpret_cast<uint4*>(dst)[j] = make_uint4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < t.n) dst[j] = __uint_as_float(r[j]);
      }
    }
  }
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(ps->cta == 0 ? &ps->acc_empty[b] : &ps->pdrained[b]);
  return true;
}

// Leader CTA, one lane of the MMA warp: pair tile t into accumulator
// (tile_no & 1) once both CTAs drained it, from the k-steps both stage.
__device__ __forceinline__ bool pr_mma(const FzTile& t, uint8_t* stages, PrShared* ps, uint32_t it,
                                       uint32_t tile_no, uint64_t timeout_ns, volatile uint32_t* cta_abort,
                                       uint32_t* fail_where, uint64_t* wait_acc) {
  const uint32_t b = tile_no & 1u;
  if (!mbar_wait_cluster(&ps->acc_empty[b], ((tile_no >> 1) & 1u) ^ 1u, timeout_ns, cta_abort)) {
    *fail_where = kWhereAccumBarrier;
    *cta_abort = 1;
    return false;
  }
  tc_fence_after();
  const uint32_t tmem = ps->tmem_base + b * kTcN;
  const int nkb = (t.k + kTcBK - 1) / kTcBK;
  for (int kb = 0; kb < nkb; ++kb) {
    const uint32_t q = it + (uint32_t)kb, s = q % ps->nstages, ph = (q / ps->nstages) & 1u;
    const uint64_t t0 = wait_acc ? globaltimer() : 0;
    if (!mbar_wait_cluster(&ps->full[s], ph, timeout_ns, cta_abort)) {
      *fail_where = kWhereFullBarrier;
      *cta_abort = 1;
      return false;
    }
    if (wait_acc) *wait_acc += globaltimer() - t0;
    tc_fence_after();
    const uint32_t sb = smem_u32(stages + s * kPrStageBytes);
    const uint64_t dAh = sdesc_k64b(sb + kPrAOff), dAl = sdesc_k64b(sb + kPrAlOff);
    const uint64_t dBh = sdesc_mn64b_pair(sb + kPrBOff), dBl = sdesc_mn64b_pair(sb + kPrBlOff);
#pragma unroll
    for (int kk = 0; kk < kTcBK / 16; ++kk) {
      const uint64_t adv_a = (uint64_t)(kk * 32) >> 4;
      const uint64_t adv_b = (uint64_t)(kk * 2 * kPrBAtomK) >> 4;
      umma_bf16_pair(tmem, dAl + adv_a, dBh + adv_b, kPrIdesc, (kb | kk) ? 1u : 0u);
      umma_bf16_pair(tmem, dAh + adv_a, dBl + adv_b, kPrIdesc, 1u);
      umma_bf16_pair(tmem, dAh + adv_a, dBh + adv_b, kPrIdesc, 1u);
    }
    umma_commit_pair(&ps->empty[s]);
  }
  umma_commit_pair(&ps->acc_full[b]);
  return true;
}

}  // namespace gvm
