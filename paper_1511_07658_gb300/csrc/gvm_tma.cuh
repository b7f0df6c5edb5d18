// Split3 SGEMM on 128 x 256 tiles whose binary32 operands arrive by TMA and
// are split in place ("TMA form").
//
// The fused form's staging warps load a k-step of A and B into registers,
// one k-step ahead, so a CTA has about 96 KB of operand loads in flight and
// the load latency sets its rate. Here a producer warp asks the tensor-copy
// unit for each k-step as soon as a stage is free -- up to all four stages,
// 192 KB, ahead of the MMAs -- and the converting warps split what has
// landed where it lies.
//
// Stage layout (48 KB, four stages, the fused form's size): a k-step of A
// is one TMA box of 128 rows x 32 binary32 values, landing as 128-byte rows
// (row r at 128 r, its 16-byte chunks swizzled: chunk j at j ^ (r % 8)); a
// k-step of B is eight slabs of 32 k-rows x 32 columns, slab c at
// 16 KB + 4 KB c (k-row kr at 128 kr inside it, swizzled alike), landed by
// one 3D box when n is a multiple of 32 and by eight 2D boxes otherwise. So every 8 rows of A and
// every 8 k-rows x 32 columns of B occupy 1 KB of their own: an atom. A warp
// converts an atom in place: all lanes read its 1 KB of binary32 (lane: row
// lane / 4, 8 values from column 8 (lane % 4); the swizzle spreads a warp's
// reads over all banks), then write the bf16 hi plane
// into its first 512 bytes and the lo plane into its last 512, each in the
// 64-byte-swizzled 8-row layout the MMA descriptors read. The descriptors
// step 1 KB between 8-row groups (A K-major; B's k groups) and 4 KB between
// B's 32-column blocks.
//
// Tasks without tensor maps (rows of A or B not 16-byte multiples, or bases
// not 16-byte aligned) are staged into the same layout by the converting
// warps' own bounds-checked loads; the producer only hands them the stage.
//
// CTA roles (kTmThreads = 352): warps 0-7 convert (two groups of four
// warps, alternate k-steps) and drain accumulators, warp 8 issues the MMAs
// (two TMEM accumulators, as in the fused form), warp 9 claims tiles, warp
// 10 produces stages. Every element of C is computed as in the other
// split3 forms: bitwise the same result.
#pragma once

#include "gvm_fused.cuh"

namespace gvm {

constexpr int kTmProducerWarp = 10;
constexpr int kTmThreads = 11 * 32;
constexpr uint32_t kTmAtom = 1024;                       // bytes of one 8-row atom (binary32 or hi + lo)
constexpr uint32_t kTmBOff = kTcM * kTcBK * 4;           // B's eight boxes start after A's 16 KB
constexpr uint32_t kTmBBox = kTcBK * 32 * 4;             // one B box: 32 k-rows x 32 columns
constexpr uint32_t kTmAtoms = (kTcM + kTcN) * kTcBK * 4 / kTmAtom;  // 48 atoms a k-step
constexpr uint32_t kTmStageTx = (kTcM + kTcN) * kTcBK * 4;          // 48 KB of boxes a k-step
constexpr int kTmBatch = 4;  // atoms a converter warp reads before it writes (12 = 3 batches a k-step)
static_assert(kTmAtoms % (kFzGroupWarps * kTmBatch) == 0, "whole batches");
static_assert(kTmStageTx == kTcStageBytes, "TMA form stage = fused stage");

struct TmShared {
  FzShared fz;                 // full / empty / accumulator barriers and TMEM, as in the fused form
  uint64_t landed[kTcStages];  // producer -> converters: the k-step's boxes landed (or the stage is free)
};

__device__ __forceinline__ void tm_init(TmShared* ts) {
  if (threadIdx.x == 0)
    for (int s = 0; s < kTcStages; ++s) mbar_init(&ts->landed[s], 1);
  fz_init(&ts->fz);  // initialises the rest, fences the inits, allocates TMEM, syncs the CTA
}

// Shared-memory descriptors of the TMA form's planes (64-byte swizzle).
// A, K-major: 8-row groups 1 KB apart.
__device__ __forceinline__ uint64_t tm_desc_a(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused when swizzled)
  d |= (uint64_t)(kTmAtom >> 4) << 32;      // stride byte offset: the next 8 rows
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}
// B, MN-major: 32-column blocks 4 KB apart (leading), 8-row k groups 1 KB
// apart (stride).
__device__ __forceinline__ uint64_t tm_desc_b(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(kTmBBox >> 4) << 16;
  d |= (uint64_t)(kTmAtom >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Global position of lane (r = lane / 4, c = lane % 4) of atom a (0..47) of
// k-step kb of tile t: 8 consecutive values of one row of A (atoms 0..15)
// or of one k-row of B (atoms 16..47: box a / 4 - 4, k group a % 4).
__device__ __forceinline__ void tm_atom_load(const FzTile& t, int kb, int a, int lane, float (&v)[8]) {
  const int r = lane >> 2, c = lane & 3;
  if (a < 16) {
    const int row = t.tm * kTcM + 8 * a + r;
    const int kk = kb * kTcBK + 8 * c;
    const float* src = t.A + (int64_t)row * t.k + kk;
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (row < t.m && kk + e < t.k) ? __ldcg(src + e) : 0.f;
  } else {
    const int box = (a - 16) >> 2, g = (a - 16) & 3;
    const int kk = kb * kTcBK + 8 * g + r;
    const int64_t col = (int64_t)t.tn * kTcN + 32 * box + 8 * c;
    const float* src = t.B + (int64_t)kk * t.n + col;
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = (kk < t.k && col + e < t.n) ? __ldcg(src + e) : 0.f;
  }
}

// Byte offset of atom a in a stage.
__device__ __forceinline__ uint32_t tm_atom_off(int a) {
  return a < 16 ? (uint32_t)a * kTmAtom : kTmBOff + (uint32_t)((a - 16) >> 2) * kTmBBox + (uint32_t)((a - 16) & 3) * kTmAtom;
}

// Converter warps: stage the k-steps of tile t that belong to this warp's
// group (k-step q of the pipeline goes to group q % 2; `it` counts the
// k-steps before this tile). landed: the tile's boxes arrive by TMA and are
// split in place; otherwise the warps load the values themselves. Warp w of
// a group takes atoms w + 4 i of each third of the k-step (A's 16 atoms,
// then B's boxes 0-3 and 4-7: atom w of box i + 4 (third - 1)), reading a
// third's four atoms before writing them. Returns false when a wait ran out
// (*cta_abort set).
__device__ __forceinline__ bool tm_convert(const FzTile& t, uint8_t* stages, TmShared* ts, uint32_t it, bool landed,
                                           uint64_t timeout_ns, volatile uint32_t* cta_abort, uint32_t* fail_where,
                                           uint64_t* wait_acc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int par = warp / kFzGroupWarps, w = warp % kFzGroupWarps;
  const int nkb = (t.k + kTcBK - 1) / kTcBK;
  const int r = lane >> 2, c = lane & 3;
  // The boxes land with the 128-byte swizzle: 16-byte chunk j of row r sits
  // at chunk j ^ r. A lane's two chunks (values 8c .. 8c+7 of row r):
  const uint32_t rd0 = (uint32_t)r * 128u + (((uint32_t)(2 * c) ^ (uint32_t)r) << 4);
  const uint32_t rd1 = (uint32_t)r * 128u + (((uint32_t)(2 * c + 1) ^ (uint32_t)r) << 4);
  const uint32_t wr = swz64((uint32_t)r, (uint32_t)c);
  const uint32_t base0 = smem_u32(stages);
  for (int kb = (int)((it + (uint32_t)par) & 1u); kb < nkb; kb += 2) {
    const uint32_t q = it + (uint32_t)kb, s = q % kTcStages, ph = (q / kTcStages) & 1u;
    uint64_t t0 = 0;
    if (wait_acc != nullptr && warp == 0 && lane == 0) t0 = globaltimer();
    if (!mbar_wait(&ts->landed[s], ph, timeout_ns, cta_abort)) {
      if (lane == 0) {
        *fail_where = kWhereEmptyBarrier;
        *cta_abort = 1;
      }
      return false;
    }
    if (t0) *wait_acc += globaltimer() - t0;
    const uint32_t st = base0 + s * kTcStageBytes;
    if (landed) {
#pragma unroll
      for (int third = 0; third < 3; ++third) {
        uint4 x[kTmBatch][2];
#pragma unroll
        for (int i = 0; i < kTmBatch; ++i) {
          const uint32_t at = st + (third == 0 ? (uint32_t)(w + 4 * i) * kTmAtom
                                               : kTmBOff + (uint32_t)(i + 4 * (third - 1)) * kTmBBox + (uint32_t)w * kTmAtom);
          x[i][0] = ld_shared_v4(at + rd0);
          x[i][1] = ld_shared_v4(at + rd1);
        }
        __syncwarp();  // every lane has read these atoms' binary32 before any lane overwrites them
#pragma unroll
        for (int i = 0; i < kTmBatch; ++i) {
          const uint32_t at = st + (third == 0 ? (uint32_t)(w + 4 * i) * kTmAtom
                                               : kTmBOff + (uint32_t)(i + 4 * (third - 1)) * kTmBBox + (uint32_t)w * kTmAtom);
          const float v[8] = {__uint_as_float(x[i][0].x), __uint_as_float(x[i][0].y), __uint_as_float(x[i][0].z),
                              __uint_as_float(x[i][0].w), __uint_as_float(x[i][1].x), __uint_as_float(x[i][1].y),
                              __uint_as_float(x[i][1].z), __uint_as_float(x[i][1].w)};
          uint4 hi, lo;
          split8_x2(v, hi, lo);
          st_shared_v4(at + wr, hi);
          st_shared_v4(at + 512u + wr, lo);
        }
      }
    } else {
      for (int j = 0; j < (int)(kTmAtoms / kFzGroupWarps); ++j) {
        const int a = j < 4 ? w + 4 * j : 16 + 4 * (j - 4) + w;
        float v[8];
        tm_atom_load(t, kb, a, lane, v);
        uint4 hi, lo;
        split8_x2(v, hi, lo);
        const uint32_t at = st + tm_atom_off(a);
        st_shared_v4(at + wr, hi);
        st_shared_v4(at + 512u + wr, lo);
      }
    }
    fence_proxy_async_shared();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ts->fz.full[s]);
  }
  return true;
}

// Producer warp, one lane: hand every k-step of tile t its stage once the
// MMAs have released it -- with the TMA boxes of A and B when the task has
// maps (tmA, tmB non-null; b3: tmB lands all eight B slabs in one 3D box),
// else as a free stage for the converters to fill.
// pend[s] records the parity of a landing still possibly in flight in stage s
// (bit 1 set), for tm_quiesce. Returns false when a wait ran out.
__device__ __forceinline__ bool tm_produce(const FzTile& t, uint8_t* stages, TmShared* ts, uint32_t it,
                                           const CUtensorMap* tmA, const CUtensorMap* tmB, bool b3, uint64_t timeout_ns,
                                           volatile uint32_t* cta_abort, uint32_t* fail_where, uint32_t* pend) {
  const int nkb = (t.k + kTcBK - 1) / kTcBK;
  const uint32_t base0 = smem_u32(stages);
  for (int kb = 0; kb < nkb; ++kb) {
    const uint32_t q = it + (uint32_t)kb, s = q % kTcStages, ph = (q / kTcStages) & 1u;
    if (!mbar_wait(&ts->fz.empty[s], ph ^ 1u, timeout_ns, cta_abort)) {
      *fail_where = kWhereEmptyBarrier;
      *cta_abort = 1;
      return false;
    }
    if (tmA != nullptr) {
      const uint32_t st = base0 + s * kTcStageBytes;
      mbar_expect_tx(&ts->landed[s], kTmStageTx);
      tma_load_2d(st, tmA, kb * kTcBK, t.tm * kTcM, &ts->landed[s]);
      if (b3) {
        tma_load_3d(stages + s * kTcStageBytes + kTmBOff, tmB, 0, kb * kTcBK, t.tn * (kTcN / 32), &ts->landed[s]);
      } else {
#pragma unroll
        for (int b = 0; b < kTcN / 32; ++b)
          tma_load_2d(st + kTmBOff + (uint32_t)b * kTmBBox, tmB, t.tn * kTcN + 32 * b, kb * kTcBK, &ts->landed[s]);
      }
      pend[s] = 2u | ph;
    } else {
      mbar_arrive(&ts->landed[s]);
      pend[s] = 0;
    }
  }
  return true;
}

// Producer lane at exit: wait (bounded, whatever the abort flag says) for
// every landing it issued, so that no tensor copy writes shared memory after
// the CTA exits.
__device__ __forceinline__ void tm_quiesce(TmShared* ts, const uint32_t* pend, uint64_t timeout_ns) {
  volatile uint32_t never = 0;
  for (int s = 0; s < kTcStages; ++s)
    if (pend[s] & 2u) (void)mbar_wait(&ts->landed[s], pend[s] & 1u, timeout_ns, &never);
}

// One elected lane of the MMA warp: tile t into accumulator (tile_no & 1),
// as fz_mma, with the TMA form's descriptors.
__device__ __forceinline__ bool tm_mma(const FzTile& t, uint8_t* stages, TmShared* ts, uint32_t it, uint32_t tile_no,
                                       uint64_t timeout_ns, volatile uint32_t* cta_abort, uint32_t* fail_where,
                                       uint64_t* wait_acc) {
  FzShared* fs = &ts->fz;
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
    const uint64_t dAh = tm_desc_a(sb), dAl = tm_desc_a(sb + 512u);
    const uint64_t dBh = tm_desc_b(sb + kTmBOff), dBl = tm_desc_b(sb + kTmBOff + 512u);
#pragma unroll
    for (int kk = 0; kk < kTcBK / 16; ++kk) {
      const uint64_t adv_a = (uint64_t)(kk * 32) >> 4;            // 16 bf16 = 32 bytes along a K-major row
      const uint64_t adv_b = (uint64_t)(kk * 2 * kTmAtom) >> 4;   // two 8-row k groups of B
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
