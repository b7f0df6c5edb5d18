// Split3 SGEMM with the split fused into operand staging, on 256 x 256 tiles
// of one CTA ("wide" tiles).
//
// The arithmetic is the fused form's (gvm_fused.cuh): per 16-wide k slice
// AlBh, AhBl, AhBh into one fp32 TMEM accumulator, k in order, so every
// element of C is bitwise the same as with 128 x 256 tiles. What changes is
// the work per staged byte: a k-step stages A (256 x 32) and B (32 x 256)
// and feeds 2 x 3 MMAs of 128 x 256 x 16 per k slice (the two 128-row halves
// of A share the B stage), twice the MMA work of a 128 x 256 tile for 4/3 of
// its operand bytes. The staging warps are bound by load latency (one k-step
// of loads per thread in flight), so more work per k-step is more work per
// latency.
//
// The accumulator of a 256 x 256 tile is all of TMEM (512 columns: rows
// 0..127 in columns 0..255, rows 128..255 in 256..511), so there is one
// accumulator: the converters drain tile T-1 right after staging their first
// k-step of tile T, and the MMAs of tile T start once it is drained.
//
// CTA roles as in the fused form (10 warps: 8 converters in two groups, MMA,
// control). On interior tiles the A operand arrives by TMA: each group owns a
// landing buffer for its k-steps' binary32 A rows (256 rows x 128 bytes),
// filled by one cp.async.bulk.tensor box of the task's A tensor map (or,
// without a map, by 256 row copies of cp.async.bulk) issued by the group's
// first warp while the group converts; the converters read A from it and
// keep only B's 64 floats of loads in registers. With all of A
// and B in registers (ragged tiles) a converter holds 128 floats of loads;
// with 10 warps a thread has at most 168 registers, so part of that spills.
//
// Stage layout (64 KB, two stages: group g fills stage g): A hi, A lo [256
// rows][32 k] K-major with the 64-byte swizzle on 8-row atoms (rows 128..255
// start 8 KB in, where the second MMA half's descriptor points); B hi, B lo
// [32 k][256 n] MN-major, as in the fused form. Then the two landing
// buffers: row r at 128 r (a warp reads 8 rows; odd rows take their second
// 16 bytes first, which spreads the reads over all banks).
#pragma once

#include "gvm_fused.cuh"

namespace gvm {

constexpr int kWdM = 256;
constexpr int kWdN = 256;
constexpr int kWdStages = 2;
constexpr uint32_t kWdAOff = 0;                       // A hi [256][32] bf16
constexpr uint32_t kWdAlOff = kWdM * kTcBK * 2;       // A lo
constexpr uint32_t kWdBOff = 2 * kWdM * kTcBK * 2;    // B hi [32][256] bf16, MN-major
constexpr uint32_t kWdBlOff = kWdBOff + kWdN * kTcBK * 2;  // B lo
constexpr uint32_t kWdStageBytes = kWdBlOff + kWdN * kTcBK * 2;
static_assert(kWdStageBytes == 65536, "wide stage layout");
constexpr uint32_t kWdHalfA = 128 * kTcBK * 2;  // bytes of 128 rows of an A plane
constexpr uint32_t kWdTmemCols = 512;
constexpr uint32_t kWdLandPitch = kTcBK * 4;                  // bytes per landed A row (dense, as TMA writes)
constexpr uint32_t kWdLandBytes = kWdM * kWdLandPitch;         // one group's landing buffer
constexpr uint32_t kWdLandTx = kWdM * kTcBK * 4;               // bytes a landing receives
constexpr uint32_t kWdSmemBytes = kWdStages * kWdStageBytes + 2 * kWdLandBytes;  // dynamic, before alignment
static_assert(kWdSmemBytes + 1024 <= 227 * 1024, "wide form shared memory");
struct WdShared {
  uint64_t full[kWdStages];   // converters -> MMA: one arrival per warp of a group
  uint64_t empty[kWdStages];  // MMA -> converters: tcgen05.commit
  uint64_t acc_full;          // MMA -> epilogue: the accumulator holds a finished tile
  uint64_t acc_empty[2];      // epilogue -> MMA: half h (rows 128 h ..) drained, one arrival per converter warp
  uint64_t land_full[2];      // bulk copies -> group g: its landing holds a k-step of A (expect_tx)
  uint64_t land_empty[2];     // group g's 4 warps -> its first warp: the landing has been read
  uint32_t tmem_base;
  uint32_t pad;
};

__device__ __forceinline__ void wd_init(WdShared* ws) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kWdStages; ++s) {
      mbar_init(&ws->full[s], kFzGroupWarps);
      mbar_init(&ws->empty[s], 1);
    }
    mbar_init(&ws->acc_full, 1);
    mbar_init(&ws->acc_empty[0], kFzConvWarps);
    mbar_init(&ws->acc_empty[1], kFzConvWarps);
    for (int g = 0; g < 2; ++g) {
      mbar_init(&ws->land_full[g], 1);
      mbar_init(&ws->land_empty[g], kFzGroupWarps);
    }
    mbar_fence_init();
  }
  if ((threadIdx.x >> 5) == kFzMmaWarp) tmem_alloc(&ws->tmem_base, kWdTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ __forceinline__ void wd_teardown(WdShared* ws) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == kFzMmaWarp) tmem_dealloc(ws->tmem_base, kWdTmemCols);
}

// Bulk copy of `bytes` (a multiple of 16) from global memory into this CTA's
// shared memory, counted on `bar` (complete_tx); both addresses 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Thread (w, lane) of a group stages k-step kb of a wide tile:
//   A item j (j = 0..7): row 8 w + (lane >> 2) + 32 j, 8 values from k = 32 kb + 8 (lane & 3);
//   B item j (j = 0..7): as in the fused form (k = 32 kb + 8 (j >> 1) + (lane >> 2),
//                        columns 32 (2 w + (j & 1)) + 8 (lane & 3)).
// Out-of-range elements are 0 (ragged m, n, k).
__device__ __forceinline__ void wd_load_a(const FzTile& t, int kb, int w, int lane, int j, int avec,
                                          float (&v)[8]) {
  const int r = t.tm * kWdM + 8 * w + (lane >> 2) + 32 * j;
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

__device__ __forceinline__ void wd_load_b(const FzTile& t, int kb, int w, int lane, int j, int bvec,
                                          float (&v)[8]) {
  const int kk = kb * kTcBK + 8 * (j >> 1) + (lane >> 2);
  const int64_t c = (int64_t)t.tn * kWdN + 32 * (2 * w + (j & 1)) + 8 * (lane & 3);
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

// Converter warps: stage the k-steps of wide tile t that belong to this
// warp's group, loads one group k-step ahead and issued after each stage's
// proxy fence (as the scheduler's fused form). after_first() runs once,
// after the group's first k-step of the tile (the previous tile's drain).
// kATma: A arrives in the group's landing buffer (a TMA box of the task's A
// map, rows and k beyond A zero-filled; without a map, row copies, interior
// tiles only); land_n / land_iss count the landings this group has consumed
// and issued (the same in all its threads). kBFast (B columns inside B, k a
// multiple of kTcBK, 32-byte aligned rows): B by unchecked 32-byte loads.
// Returns false when a wait ran out (*cta_abort set).
template <bool kATma, bool kBFast, class AfterFirst>
__device__ __forceinline__ bool wd_convert_loop(const FzTile& t, uint32_t base, WdShared* ws, uint32_t it,
                                                int avec, int bvec, uint64_t timeout_ns,
                                                volatile uint32_t* cta_abort, uint32_t* fail_where,
                                                uint64_t* wait_acc, AfterFirst& after_first, uint32_t& land_n,
                                                uint32_t& land_iss, const CUtensorMap* tmA) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int par = warp / kFzGroupWarps, w = warp % kFzGroupWarps;
  const int nkb = (t.k + kTcBK - 1) / kTcBK;
  const int kb0 = (int)((it + (uint32_t)par) & 1u);
  if (kb0 >= nkb) return true;
  const float* pb = t.B + (int64_t)(lane >> 2) * t.n + (int64_t)t.tn * kWdN + 64 * w + 8 * (lane & 3);
  const int64_t b_row8 = 8 * t.n, b_step = (int64_t)kTcBK * t.n;
  const uint32_t land = base + kWdStages * kWdStageBytes + (uint32_t)par * kWdLandBytes;
  auto fail = [&](uint32_t where) {
    if (lane == 0) {
      *fail_where = where;
      *cta_abort = 1;
    }
    return false;
  };
  // The group's first warp refills the landing with k-step kb's A rows once
  // all four warps have read the previous landing.
  auto land_a = [&](int kb) -> bool {
    if (w != 0) return true;
    if (land_n > 0 && !mbar_wait(&ws->land_empty[par], (land_n - 1) & 1u, timeout_ns, cta_abort))
      return fail(kWhereEmptyBarrier);
    if (lane == 0) mbar_expect_tx(&ws->land_full[par], kWdLandTx);
    __syncwarp();
    if (tmA != nullptr) {
      if (lane == 0) tma_load_2d(land, tmA, kb * kTcBK, t.tm * kWdM, &ws->land_full[par]);
    } else {
      const float* src = t.A + (int64_t)(t.tm * kWdM) * t.k + kb * kTcBK;
#pragma unroll
      for (int i = 0; i < kWdM / 32; ++i) {
        const int r = lane + 32 * i;
        bulk_g2s(land + (uint32_t)r * kWdLandPitch, src + (int64_t)r * t.k, kTcBK * 4, &ws->land_full[par]);
      }
    }
    ++land_iss;
    return true;
  };
  auto load_a = [&](int kb, int j, float (&v)[8]) { wd_load_a(t, kb, w, lane, j, avec, v); };
  auto load_b = [&](int kb, int j, float (&v)[8]) {
    if (kBFast) ld_cg_v8(pb + kb * b_step + (j >> 1) * b_row8 + 32 * (j & 1), v);
    else wd_load_b(t, kb, w, lane, j, bvec, v);
  };
  float va[kATma ? 1 : 8][8], vb[8][8];
  if (kATma) {
    if (!land_a(kb0)) return false;
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) load_a(kb0, j, va[kATma ? 0 : j]);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) load_b(kb0, j, vb[j]);
  const uint32_t a_off = (uint32_t)(8 * w) * 64u + swz64((uint32_t)(lane >> 2), (uint32_t)(lane & 3));
  const uint32_t b_off = swz64((uint32_t)(lane >> 2), (uint32_t)(lane & 3));
  // A item j of this thread in the landing: row 8 w + (lane >> 2) + 32 j, bytes 32 (lane & 3) ..
  const uint32_t a_land = land + (uint32_t)(8 * w + (lane >> 2)) * kWdLandPitch + 32u * (uint32_t)(lane & 3);
  bool first = true;
  for (int kb = kb0; kb < nkb; kb += 2) {
    const uint32_t q = it + (uint32_t)kb, s = q % kWdStages, ph = (q / kWdStages) & 1u;
    uint64_t t0 = 0;
    if (wait_acc != nullptr && warp == 0 && lane == 0) t0 = globaltimer();
    if (!mbar_wait(&ws->empty[s], ph ^ 1u, timeout_ns, cta_abort)) return fail(kWhereEmptyBarrier);
    if (kATma) {
      if (!mbar_wait(&ws->land_full[par], land_n & 1u, timeout_ns, cta_abort)) return fail(kWhereFullBarrier);
      ++land_n;
    }
    if (t0) *wait_acc += globaltimer() - t0;
    const uint32_t st = base + s * kWdStageBytes;
    const bool more = kb + 2 < nkb;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      // Row 8 w + (lane >> 2) + 32 j: its swizzle phase depends on the row
      // within its 8-row atom only, so every j shares a_off.
      const uint32_t off = a_off + (uint32_t)(32 * j) * 64u;
      uint4 hi, lo;
      if (kATma) {
        // Odd rows of the 8 read their second 16 bytes first: the warp's
        // 32 reads then fall on 8 different bank groups.
        const uint32_t ra = a_land + (uint32_t)(32 * j) * kWdLandPitch;
        const uint32_t sw = ((lane >> 2) & 1) ? 16u : 0u;
        const uint4 x0 = ld_shared_v4(ra + sw), x1 = ld_shared_v4(ra + (sw ^ 16u));
        const uint4 lo4 = sw ? x1 : x0, hi4 = sw ? x0 : x1;
        float v[8] = {__uint_as_float(lo4.x), __uint_as_float(lo4.y), __uint_as_float(lo4.z),
                      __uint_as_float(lo4.w), __uint_as_float(hi4.x), __uint_as_float(hi4.y),
                      __uint_as_float(hi4.z), __uint_as_float(hi4.w)};
        split8_x2(v, hi, lo);
      } else {
        split8_x2(va[kATma ? 0 : j], hi, lo);
      }
      st_shared_v4(st + kWdAOff + off, hi);
      st_shared_v4(st + kWdAlOff + off, lo);
    }
    if (kATma) {
      // This warp has read its rows of the landing.
      __syncwarp();
      if (lane == 0) mbar_arrive(&ws->land_empty[par]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t off = (uint32_t)(j >> 1) * kFzBAtomK + (uint32_t)(2 * w + (j & 1)) * kFzBAtomN + b_off;
      uint4 hi, lo;
      split8_x2(vb[j], hi, lo);
      st_shared_v4(st + kWdBOff + off, hi);
      st_shared_v4(st + kWdBlOff + off, lo);
    }
    fence_proxy_async_shared();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ws->full[s]);
    if (more) {
      if (kATma) {
        if (!land_a(kb + 2)) return false;
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) load_a(kb + 2, j, va[kATma ? 0 : j]);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) load_b(kb + 2, j, vb[j]);
    }
    if (first) {
      first = false;
      if (!after_first()) return false;
    }
  }
  return true;
}

// The variants other than the interior one in functions of their own, so
// that their register needs do not weigh on the interior tiles' loop.
template <bool kATma, class AfterFirst>
__device__ __noinline__ bool wd_convert_ragged(const FzTile& t, uint32_t base, WdShared* ws, uint32_t it, int avec,
                                               int bvec, uint64_t timeout_ns, volatile uint32_t* cta_abort,
                                               uint32_t* fail_where, uint64_t* wait_acc, AfterFirst& after_first,
                                               uint32_t& land_n, uint32_t& land_iss, const CUtensorMap* tmA) {
  return wd_convert_loop<kATma, false>(t, base, ws, it, avec, bvec, timeout_ns, cta_abort, fail_where, wait_acc,
                                       after_first, land_n, land_iss, tmA);
}

template <class AfterFirst>
__device__ __forceinline__ bool wd_convert(const FzTile& t, uint8_t* stages, WdShared* ws, uint32_t it,
                                           uint64_t timeout_ns, volatile uint32_t* cta_abort,
                                           uint32_t* fail_where, uint64_t* wait_acc, AfterFirst after_first,
                                           uint32_t& land_n, uint32_t& land_iss, const CUtensorMap* tmA = nullptr) {
  const int avec = ((t.k & 7) == 0 && (reinterpret_cast<uintptr_t>(t.A) & 31) == 0)   ? 2
                   : ((t.k & 3) == 0 && (reinterpret_cast<uintptr_t>(t.A) & 15) == 0) ? 1
                                                                                      : 0;
  const int bvec = ((t.n & 7) == 0 && (reinterpret_cast<uintptr_t>(t.B) & 31) == 0)   ? 2
                   : ((t.n & 3) == 0 && (reinterpret_cast<uintptr_t>(t.B) & 15) == 0) ? 1
                                                                                      : 0;
  const bool interior = avec == 2 && (t.tm + 1) * kWdM <= t.m;  // A rows by row copies without a map
  const bool b_fast = bvec == 2 && (t.k % kTcBK) == 0 && (int64_t)(t.tn + 1) * kWdN <= t.n;
  const uint32_t base = smem_u32(stages);
  if (b_fast && (tmA != nullptr || (interior && (t.k % kTcBK) == 0)))
    return wd_convert_loop<true, true>(t, base, ws, it, avec, bvec, timeout_ns, cta_abort, fail_where, wait_acc,
                                       after_first, land_n, land_iss, tmA);
  if (tmA != nullptr)
    return wd_convert_ragged<true>(t, base, ws, it, avec, bvec, timeout_ns, cta_abort, fail_where, wait_acc,
                                   after_first, land_n, land_iss, tmA);
  return wd_convert_ragged<false>(t, base, ws, it, avec, bvec, timeout_ns, cta_abort, fail_where, wait_acc,
                                  after_first, land_n, land_iss, nullptr);
}

// Converter warps, once they stop (normally every landing issued has been
// consumed; after a failed wait one may still be in flight): wait, bounded
// and whatever the abort flag says, for the group's last issued landing, so
// that no bulk copy writes this CTA's shared memory after it exits.
__device__ __forceinline__ void wd_land_quiesce(WdShared* ws, uint32_t land_n, uint32_t land_iss,
                                                uint64_t timeout_ns) {
  const int par = (threadIdx.x >> 5) / kFzGroupWarps;
  if (land_iss <= land_n) return;
  volatile uint32_t never = 0;
  (void)mbar_wait(&ws->land_full[par], (land_iss - 1) & 1u, timeout_ns, &never);
}

// Converter warps: drain the accumulator of wide tile t (the tile_no-th of
// this CTA) into C. Warp w reads TMEM lanes 32 (w & 3) .. +31 of both halves
// (rows 32 (w & 3) + lane and 128 + 32 (w & 3) + lane of the tile), columns
// 128 (w >> 2) .. +127 of each half, 32 at a time, and stores whole 32-byte
// sectors (16-byte or single stores when n does not allow). Then frees the
// accumulator.
__device__ __forceinline__ bool wd_epilogue(const FzTile& t, WdShared* ws, uint32_t tile_no, uint64_t timeout_ns,
                                            volatile uint32_t* cta_abort, uint32_t* fail_where) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!mbar_wait(&ws->acc_full, tile_no & 1u, timeout_ns, cta_abort)) {
    if (lane == 0) {
      *fail_where = kWhereAccumBarrier;
      *cta_abort = 1;
    }
    return false;
  }
  tc_fence_after();
  const int q = warp & 3, cq = warp >> 2;
  const uintptr_t ca = reinterpret_cast<uintptr_t>(t.C);
  const int vec = ((t.n & 7) == 0 && (ca & 31) == 0) ? 2 : ((t.n & 3) == 0 && (ca & 15) == 0) ? 1 : 0;
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    const int row = t.tm * kWdM + h * 128 + q * 32 + lane;
#pragma unroll 1
    for (int ch = 0; ch < 4; ++ch) {
      const int chunk = cq * 4 + ch;
      uint32_t r[32];
      tmem_ld_32x32b_x32(ws->tmem_base + (uint32_t)(h * kWdN) + ((uint32_t)(q * 32) << 16) + (uint32_t)(chunk * 32),
                         r);
      tmem_ld_wait();
      const int64_t c0 = (int64_t)t.tn * kWdN + chunk * 32;
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
    // Half h is drained: the next tile's MMAs into it may start while the
    // other half drains.
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ws->acc_empty[h]);
  }
  return true;
}

// One elected lane of the MMA warp: accumulate wide tile t (the tile_no-th
// of this CTA) once the previous tile's accumulator has been drained.
__device__ __forceinline__ bool wd_mma(const FzTile& t, uint8_t* stages, WdShared* ws, uint32_t it,
                                       uint32_t tile_no, uint64_t timeout_ns, volatile uint32_t* cta_abort,
                                       uint32_t* fail_where, uint64_t* wait_acc) {
  // Half 0 of the accumulator must be drained before the first MMA; half 1
  // is waited for inside the first k-step, before its first MMA.
  if (!mbar_wait(&ws->acc_empty[0], (tile_no & 1u) ^ 1u, timeout_ns, cta_abort)) {
    *fail_where = kWhereAccumBarrier;
    *cta_abort = 1;
    return false;
  }
  tc_fence_after();
  const int nkb = (t.k + kTcBK - 1) / kTcBK;
  for (int kb = 0; kb < nkb; ++kb) {
    const uint32_t q = it + (uint32_t)kb, s = q % kWdStages, ph = (q / kWdStages) & 1u;
    const uint64_t t0 = wait_acc ? globaltimer() : 0;
    if (!mbar_wait(&ws->full[s], ph, timeout_ns, cta_abort)) {
      *fail_where = kWhereFullBarrier;
      *cta_abort = 1;
      return false;
    }
    if (wait_acc) *wait_acc += globaltimer() - t0;
    tc_fence_after();
    const uint32_t sb = smem_u32(stages + s * kWdStageBytes);
    const uint64_t dBh = sdesc_mn64b(sb + kWdBOff), dBl = sdesc_mn64b(sb + kWdBlOff);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && kb == 0) {
        if (!mbar_wait(&ws->acc_empty[1], (tile_no & 1u) ^ 1u, timeout_ns, cta_abort)) {
          *fail_where = kWhereAccumBarrier;
          *cta_abort = 1;
          return false;
        }
        tc_fence_after();
      }
      const uint32_t tmem = ws->tmem_base + (uint32_t)(h * kWdN);
      const uint64_t dAh = sdesc_k64b(sb + kWdAOff + h * kWdHalfA), dAl = sdesc_k64b(sb + kWdAlOff + h * kWdHalfA);
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk) {
        const uint64_t adv_a = (uint64_t)(kk * 32) >> 4;             // 16 bf16 = 32 bytes along a K-major row
        const uint64_t adv_b = (uint64_t)(kk * 2 * kFzBAtomK) >> 4;  // two 8-row k groups of B
        umma_bf16(tmem, dAl + adv_a, dBh + adv_b, kFzIdesc, (kb | kk) ? 1u : 0u);
        umma_bf16(tmem, dAh + adv_a, dBl + adv_b, kFzIdesc, 1u);
        umma_bf16(tmem, dAh + adv_a, dBh + adv_b, kFzIdesc, 1u);
      }
    }
    umma_commit(&ws->empty[s]);
  }
  umma_commit(&ws->acc_full);
  return true;
}

}  // namespace gvm
