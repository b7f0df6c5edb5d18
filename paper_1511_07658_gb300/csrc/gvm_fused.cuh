// Split3 SGEMM with the split fused into operand staging.
//
// C = AhBh + AhBl + AlBh (hi = RN_bf16(x), lo = RN_bf16(x - hi)) on tcgen05
// tensor cores, like tc_tile, but without a pre-pass: the warps that stage a
// k-step of A and B into shared memory load the binary32 operands straight
// from global memory, split them in registers and store the bf16 hi and lo
// planes in the 64-byte-swizzled K-major layout the MMA descriptors read (the
// layout TMA writes for tc_tile). Nothing is written back to HBM but C.
//
// CTA roles (kFzThreads = 320 threads, one CTA per SM):
//   warps 0..7   converters, two groups of four warps: group g stages the
//                k-steps q with q % 2 == g, so two k-steps are in flight at
//                once. The same warps drain a finished accumulator from TMEM
//                into C (the epilogue) after staging the next tile, and run
//                vector-add tiles.
//   warp 8       MMA issue (one elected lane): per k-step 2 x 3 MMAs of
//                128 x 256 x 16 into one of two TMEM accumulators, so that the
//                epilogue of a tile overlaps the MMAs of the next one.
//   warp 9       the scheduler's tile claims (idle in the standalone kernel).
// Ten warps leave 168 registers a thread: a converter keeps a whole k-step
// share (96 floats) of loads in flight.
//
// Stage layout (kTcStageBytes = 48 KB, the byte offsets of tc_tile's stage):
//   A hi, A lo  [128 rows][32 k] K-major, like tc_tile's;
//   B hi, B lo  [32 k][256 n] MN-major (n contiguous, as B is stored), so that
//               the converters load rows of B with 16-byte loads and store
//               8-column chunks without a transpose.
// Both use the 64-byte swizzle (address bits 4-5 ^= bits 7-8) on atoms of
// 8 rows x 64 bytes. A: atom i holds rows 8i..8i+7 (stride 512 B). B: atom
// (g, b) holds k rows 8g..8g+7 and columns 32b..32b+31 at 4096 g + 512 b.
#pragma once

#include "gvm_device.cuh"

namespace gvm {

constexpr int kFzConvWarps = 8;
constexpr int kFzConvThreads = kFzConvWarps * 32;
constexpr int kFzGroupWarps = 4;
constexpr int kFzMmaWarp = 8;
constexpr int kFzCtlWarp = 9;
constexpr int kFzThreads = 10 * 32;
constexpr uint32_t kFzTmemCols = 2 * kTcN;  // two 128 x 256 fp32 accumulators
constexpr uint32_t kFzNamedBarrier = 1;     // bar.sync id of the converter warps

struct FzShared {
  uint64_t full[kTcStages];   // converters -> MMA: one arrival per warp of a group
  uint64_t empty[kTcStages];  // MMA -> converters: tcgen05.commit
  uint64_t acc_full[2];       // MMA -> epilogue: accumulator b complete
  uint64_t acc_empty[2];      // epilogue -> MMA: one arrival per converter warp
  uint32_t tmem_base;
  uint32_t pad;
};

// One GEMM tile as the converters and the MMA warp see it.
struct FzTile {
  const float* A;
  const float* B;
  float* C;
  int64_t n;
  int m;
  int k;
  int tm;
  int tn;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
  return v;
}
// Makes this thread's generic-proxy shared-memory stores visible to the
// async proxy (the tensor core reads the stage through it).
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void conv_barrier() {
  asm volatile("bar.sync %0, %1;" ::"n"(kFzNamedBarrier), "n"(kFzConvThreads) : "memory");
}

__device__ __forceinline__ uint32_t swz64(uint32_t row, uint32_t chunk) {
  return row * 64u + ((chunk ^ ((row >> 1) & 3u)) << 4);
}

// Shared-memory descriptor of an MN-major B operand (layout above): 32-column
// atoms 512 B apart along N (leading byte offset), 8-row k groups 4096 B
// apart (stride byte offset), 64-byte swizzle.
constexpr uint32_t kFzBAtomN = 512;
constexpr uint32_t kFzBAtomK = 4096;
__device__ __forceinline__ uint64_t sdesc_mn64b(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(kFzBAtomN >> 4) << 16;
  d |= (uint64_t)(kFzBAtomK >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
// Instruction descriptor: tc_tile's, with B MN-major (bit 16).
constexpr uint32_t kFzIdesc = idesc_bf16_f32(kTcM, kTcN) | (1u << 16);

// split8 with the residual x - hi taken two at a time (sub.rn.f32x2); the
// bf16 pair packs element 2i in its low half, so its binary32 value is the
// half shifted up, and element 2i+1's is the high half with the low bits
// cleared. Same values as split8, fewer instructions.
__device__ __forceinline__ void split8_x2(const float (&v)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const uint32_t hu = *reinterpret_cast<const uint32_t*>(&hb);
    const float h0 = __uint_as_float(hu << 16), h1 = __uint_as_float(hu & 0xffff0000u);
    float d0, d1;
    asm("{\n\t.reg .b64 x, y, d;\n\t"
        "mov.b64 x, {%2, %3};\n\t"
        "mov.b64 y, {%4, %5};\n\t"
        "sub.rn.f32x2 d, x, y;\n\t"
        "mov.b64 {%0, %1}, d;\n\t}"
        : "=f"(d0), "=f"(d1)
        : "f"(v[2 * i]), "f"(v[2 * i + 1]), "f"(h0), "f"(h1));
    const __nv_bfloat162 lb = __floats2bfloat162_rn(d0, d1);
    h[i] = hu;
    l[i] = *reinterpret_cast<const uint32_t*>(&lb);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void fz_init(FzShared* fs) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&fs->full[s], kFzGroupWarps);
      mbar_init(&fs->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&fs->acc_full[b], 1);
      mbar_init(&fs->acc_empty[b], kFzConvWarps);
    }
    mbar_fence_init();
  }
  if ((threadIdx.x >> 5) == kFzMmaWarp) tmem_alloc(&fs->tmem_base, kFzTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ __forceinline__ void fz_teardown(FzShared* fs) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == kFzMmaWarp) tmem_dealloc(fs->tmem_base, kFzTmemCols);
}

// 32-byte load of 8 floats (one converter item) through L2; the address must
// be 32-byte aligned.
__device__ __forceinline__ void ld_cg_v8(const float* p, float (&v)[8]) {
  asm("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "l"(p));
}

// ---------------------------------------------------------------- converters

// Thread (w, lane) of a group (w = warp index in the group, 0..3) stages k-step kb:
//   A item j (j = 0..3): row 8 w + (lane >> 2) + 32 j, 8 values from k = 32 kb + 8 (lane & 3);
//   B item j (j = 0..7): k = 32 kb + 8 (j >> 1) + (lane >> 2), 8 values from
//                        column 32 (2 w + (j & 1)) + 8 (lane & 3).
// Every load instruction of a warp reads 8 rows x 128 contiguous bytes and
// every store fills one 512-byte swizzle atom (no bank conflicts).
// Out-of-range elements are 0 (ragged m, n, k).
__device__ __forceinline__ void fz_load_a(const FzTile& t, int kb, int w, int lane, int j, int avec,
                                          float (&v)[8]) {
  const int r = t.tm * kTcM + 8 * w + (lane >> 2) + 32 * j;
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
__device__ __forceinline__ void fz_load_b(const FzTile& t, int kb, int w, int lane, int j, int bvec,
                                          float (&v)[8]) {
  const int kk = kb * kTcBK + 8 * (j >> 1) + (lane >> 2);
  const int64_t c = (int64_t)t.tn * kTcN + 32 * (2 * w + (j & 1)) + 8 * (lane & 3);
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

// Converter warps: stage every k-step of tile t that belongs to this warp's
// group. `it` is the pipeline's k-step counter before this tile (the same
// value in every role). Loads run one k-step (of this group) ahead: as soon
// as an item is split and stored, its registers take the item's next load,
// so a thread has its share of operands in flight nearly all the time
// (the stage ring alone cannot cover the load latency at this rate).
// kFast: an interior tile, k a multiple of kTcBK and 32-byte aligned rows;
// every item is one 32-byte load at a fixed offset from two per-thread bases.
// Otherwise each load checks its bounds and picks the widest access the
// alignment allows. kLate: the next k-step's loads are issued after the
// stage's proxy fence and arrive instead of between the stores (measured: the
// scheduler kernel, which interleaves tiles of many tasks, runs 7% faster so;
// the single-GEMM kernel 5% slower). Returns false when a wait ran out
// (*cta_abort set).
template <bool kFast, bool kLate>
__device__ __forceinline__ bool fz_convert_loop(const FzTile& t, uint32_t base, FzShared* fs, uint32_t it,
                                                int avec, int bvec, uint64_t timeout_ns,
                                                volatile uint32_t* cta_abort, uint32_t* fail_where,
                                                uint64_t* wait_acc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int par = warp / kFzGroupWarps, w = warp % kFzGroupWarps;
  const int nkb = (t.k + kTcBK - 1) / kTcBK;
  // First k-step of this tile with the group's parity.
  const int kb0 = (int)((it + (uint32_t)par) & 1u);
  if (kb0 >= nkb) return true;
  const float* pa = t.A + (int64_t)(t.tm * kTcM + 8 * w + (lane >> 2)) * t.k + 8 * (lane & 3);
  const float* pb = t.B + (int64_t)(lane >> 2) * t.n + (int64_t)t.tn * kTcN + 64 * w + 8 * (lane & 3);
  const int64_t a_row32 = 32 * (int64_t)t.k, b_row8 = 8 * t.n, b_step = (int64_t)kTcBK * t.n;
  auto load_a = [&](int kb, int j, float (&v)[8]) {
    if (kFast) ld_cg_v8(pa + kb * kTcBK + j * a_row32, v);
    else fz_load_a(t, kb, w, lane, j, avec, v);
  };
  auto load_b = [&](int kb, int j, float (&v)[8]) {
    if (kFast) ld_cg_v8(pb + kb * b_step + (j >> 1) * b_row8 + 32 * (j & 1), v);
    else fz_load_b(t, kb, w, lane, j, bvec, v);
  };
  float va[4][8], vb[8][8];
#pragma unroll
  for (int j = 0; j < 4; ++j) load_a(kb0, j, va[j]);
#pragma unroll
  for (int j = 0; j < 8; ++j) load_b(kb0, j, vb[j]);
  const uint32_t a_off = (uint32_t)(8 * w) * 64u + swz64((uint32_t)(lane >> 2), (uint32_t)(lane & 3));
  const uint32_t b_off = swz64((uint32_t)(lane >> 2), (uint32_t)(lane & 3));
  for (int kb = kb0; kb < nkb; kb += 2) {
    const uint32_t q = it + (uint32_t)kb, s = q % kTcStages, ph = (q / kTcStages) & 1u;
    uint64_t t0 = 0;
    if (wait_acc != nullptr && warp == 0 && lane == 0) t0 = globaltimer();
    if (!mbar_wait(&fs->empty[s], ph ^ 1u, timeout_ns, cta_abort)) {
      if (lane == 0) {
        *fail_where = kWhereEmptyBarrier;
        *cta_abort = 1;
      }
      return false;
    }
    if (t0) *wait_acc += globaltimer() - t0;
    const uint32_t st = base + s * kTcStageBytes;
    const bool more = kb + 2 < nkb;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      // Row 8 w + (lane >> 2) + 32 j: the swizzle phase depends on the row
      // within its 8-row atom only, so atom j * 4 + w shares a_off.
      const uint32_t off = a_off + (uint32_t)(32 * j) * 64u;
      uint4 hi, lo;
      split8_x2(va[j], hi, lo);
      st_shared_v4(st + kTcAOff + off, hi);
      st_shared_v4(st + kTcAlOff + off, lo);
      if (!kLate && more) load_a(kb + 2, j, va[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t off = (uint32_t)(j >> 1) * kFzBAtomK + (uint32_t)(2 * w + (j & 1)) * kFzBAtomN + b_off;
      uint4 hi, lo;
      split8_x2(vb[j], hi, lo);
      st_shared_v4(st + kTcBOff + off, hi);
      st_shared_v4(st + kTcBlOff + off, lo);
      if (!kLate && more) load_b(kb + 2, j, vb[j]);
    }
    fence_proxy_async_shared();
    __syncwarp();
    if (lane == 0) mbar_arrive(&fs->full[s]);
    if (kLate && more) {
      // The next loads go out after the proxy fence, so that the fence does
      // not hold them (or wait for them) while the stage is handed over.
#pragma unroll
      for (int j = 0; j < 4; ++j) load_a(kb + 2, j, va[j]);
#pragma unroll
      for (int j = 0; j < 8; ++j) load_b(kb + 2, j, vb[j]);
    }
  }
  return true;
}

template <bool kLate>
__device__ __forceinline__ bool fz_convert(const FzTile& t, uint8_t* stages, FzShared* fs, uint32_t it,
                                           uint64_t timeout_ns, volatile uint32_t* cta_abort,
                                           uint32_t* fail_where, uint64_t* wait_acc) {
  // Widest load every item of the tile allows: 2 = 32 bytes, 1 = 16 bytes, 0 = scalar.
  const int avec = ((t.k & 7) == 0 && (reinterpret_cast<uintptr_t>(t.A) & 31) == 0)   ? 2
                   : ((t.k & 3) == 0 && (reinterpret_cast<uintptr_t>(t.A) & 15) == 0) ? 1
                                                                                      : 0;
  const int bvec = ((t.n & 7) == 0 && (reinterpret_cast<uintptr_t>(t.B) & 31) == 0)   ? 2
                   : ((t.n & 3) == 0 && (reinterpret_cast<uintptr_t>(t.B) & 15) == 0) ? 1
                                                                                      : 0;
  const bool fast = avec == 2 && bvec == 2 && (t.k % kTcBK) == 0 && (t.tm + 1) * kTcM <= t.m &&
                    (int64_t)(t.tn + 1) * kTcN <= t.n;
  const uint32_t base = smem_u32(stages);
  return fast ? fz_convert_loop<true, kLate>(t, base, fs, it, avec, bvec, timeout_ns, cta_abort, fail_where,
                                             wait_acc)
              : fz_convert_loop<false, kLate>(t, base, fs, it, avec, bvec, timeout_ns, cta_abort, fail_where,
                                              wait_acc);
}

// 32-byte store of 8 floats; the address must be 32-byte aligned.
__device__ __forceinline__ void st_v8(float* p, const uint32_t* r) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(r[0]), "r"(r[1]), "r"(r[2]),
               "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}

// Converter warps: drain accumulator (tile_no & 1) of tile t into C. Warp w
// reads TMEM lanes 32 (w & 3) .. +31 (rows of the tile) and columns
// 128 (w >> 2) .. +127, 32 columns at a time; TMEM hands each thread one
// row, which it stores as whole 32-byte sectors (16-byte or single stores
// when n does not allow). No shared memory: the operand loads keep all of L1
// for their requests in flight. Then frees the accumulator.
__device__ __forceinline__ bool fz_epilogue(const FzTile& t, FzShared* fs, uint32_t tile_no, uint64_t timeout_ns,
                                            volatile uint32_t* cta_abort, uint32_t* fail_where) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t b = tile_no & 1u;
  if (!mbar_wait(&fs->acc_full[b], (tile_no >> 1) & 1u, timeout_ns, cta_abort)) {
    if (lane == 0) {
      *fail_where = kWhereAccumBarrier;
      *cta_abort = 1;
    }
    return false;
  }
  tc_fence_after();
  const int q = warp & 3, cq = warp >> 2;
  const int row = t.tm * kTcM + q * 32 + lane;
  const uintptr_t ca = reinterpret_cast<uintptr_t>(t.C);
  const int vec = ((t.n & 7) == 0 && (ca & 31) == 0) ? 2 : ((t.n & 3) == 0 && (ca & 15) == 0) ? 1 : 0;
  // One row's 32 columns from chunk `chunk` into C.
  auto store_chunk = [&](int chunk, const uint32_t (&r)[32]) {
    const int64_t c0 = (int64_t)t.tn * kTcN + chunk * 32;
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
  };
  // Two 32-column chunks a TMEM round trip (the staging registers are free
  // here), four chunks a warp.
  const uint32_t taddr = fs->tmem_base + b * kTcN + ((uint32_t)(q * 32) << 16);
#pragma unroll 1
  for (int ch = 0; ch < 4; ch += 2) {
    const int chunk = cq * 4 + ch;
    uint32_t r0[32], r1[32];
    tmem_ld_32x32b_x32(taddr + (uint32_t)(chunk * 32), r0);
    tmem_ld_32x32b_x32(taddr + (uint32_t)((chunk + 1) * 32), r1);
    tmem_ld_wait();
    store_chunk(chunk, r0);
    store_chunk(chunk + 1, r1);
  }
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(&fs->acc_empty[b]);
  return true;
}

// ---------------------------------------------------------------- MMA warp

// One elected lane of the MMA warp: accumulate tile t into TMEM accumulator
// (tile_no & 1) once the epilogue has drained it, consuming the k-steps the
// converters stage. Returns false when a wait ran out (*cta_abort set).
__device__ __forceinline__ bool fz_mma(const FzTile& t, uint8_t* stages, FzShared* fs, uint32_t it,
                                       uint32_t tile_no, uint64_t timeout_ns, volatile uint32_t* cta_abort,
                                       uint32_t* fail_where, uint64_t* wait_acc) {
  const uint32_t b = tile_no & 1u;
  if (!mbar_wait(&fs->acc_empty[b], ((tile_no >> 1) & 1u) ^ 1u, timeout_ns, cta_abort)) {
    *fail_where = kWhereAccumBarrier;
    *cta_abort = 1;
    return false;
  }
  tc_fence_after();
  const uint32_t tmem = fs->tmem_base + b * kTcN;
  const int nkb = (t.k + kTcBK - 1) / kTcBK;
  for (int kb = 0; kb < nkb; ++kb) {
    const uint32_t q = it + (uint32_t)kb, s = q % kTcStages, ph = (q / kTcStages) & 1u;
    const uint64_t t0 = wait_acc ? globaltimer() : 0;
    if (!mbar_wait(&fs->full[s], ph, timeout_ns, cta_abort)) {
      *fail_where = kWhereFullBarrier;
      *cta_abort = 1;
      return false;
    }
    if (wait_acc) *wait_acc += globaltimer() - t0;
    tc_fence_after();
    const uint32_t sb = smem_u32(stages + s * kTcStageBytes);
    const uint64_t dAh = sdesc_k64b(sb + kTcAOff), dAl = sdesc_k64b(sb + kTcAlOff);
    const uint64_t dBh = sdesc_mn64b(sb + kTcBOff), dBl = sdesc_mn64b(sb + kTcBlOff);
#pragma unroll
    for (int kk = 0; kk < kTcBK / 16; ++kk) {
      const uint64_t adv_a = (uint64_t)(kk * 32) >> 4;             // 16 bf16 = 32 bytes along a K-major row
      const uint64_t adv_b = (uint64_t)(kk * 2 * kFzBAtomK) >> 4;  // two 8-row k groups of B
      umma_bf16(tmem, dAl + adv_a, dBh + adv_b, kFzIdesc, (kb | kk) ? 1u : 0u);
      umma_bf16(tmem, dAh + adv_a, dBl + adv_b, kFzIdesc, 1u);
      umma_bf16(tmem, dAh + adv_a, dBh + adv_b, kFzIdesc, 1u);
    }
    umma_commit(&fs->empty[s]);
  }
  umma_commit(&fs->acc_full[b]);
  return true;
}

}  // namespace gvm
