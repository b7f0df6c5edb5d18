// Device code shared by the persistent scheduler and the standalone task
// kernels: PTX wrappers, and one function per tile kind.
//
//   vadd_range   vector-add task (Table 2, VecAdd): c = a + b, binary32
//   vmul_range   vector-multiply task (Table 2, VecMul): iterated binary32 products
//   fma_tile     matrix-multiply task (Table 2, MM) on the CUDA cores
//   split_*      split3 pre-pass: x -> (hi, lo) bf16 pair, x = hi + lo + r
//   tc_tile      split3 product AhBh + AhBl + AlBh on tcgen05 tensor cores,
//                operands staged by TMA, accumulator in TMEM
//
// Every wait is bounded by a deadline on %globaltimer; a wait that runs out
// reports failure to its caller, which records a status word and stops.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "gvm_internal.h"

namespace gvm {

// ---------------------------------------------------------------- PTX basics

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_acquire_gpu64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_acquire_sys(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_gpu64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release_gpu64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys(uint32_t* p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_sys64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// 16-byte load that bypasses L1 (data written by other CTAs or by the host).
__device__ __forceinline__ uint4 ld_cg_v4(const void* p) {
  uint4 v;
  asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
__device__ __forceinline__ uint4 ld_volatile_v4(const void* p) {
  uint4 v;
  asm volatile("ld.volatile.global.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_cg_v4(void* p, uint4 v) {
  asm volatile("st.global.cg.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_tensormap_release() {
  asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
}
__device__ __forceinline__ void fence_tensormap_acquire(const void* tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}

// ---------------------------------------------------------------- mbarrier

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity. Gives up when the
// deadline passes or another warp of the CTA has flagged an abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t timeout_ns,
                                          volatile uint32_t* cta_abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t deadline = globaltimer() + timeout_ns;
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*cta_abort) return false;
    if (globaltimer() > deadline) return false;
  }
}

// ---------------------------------------------------------------- TMA

__device__ __forceinline__ void tma_load_3d(void* smem_dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(smem_dst)),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t smem_dst, const CUtensorMap* tm, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_dst),
      "l"(tm), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------- tcgen05

__device__ __forceinline__ void tmem_alloc(uint32_t* smem_slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, bf16 inputs, fp32 accumulate, both K-major.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrives on the mbarrier once every MMA issued so far by this thread is done.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
// 32 lanes x 32 consecutive fp32 columns: thread t of the warp gets lane (base + t).
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows of
// kTcBK bf16 (64 bytes), 8-row core groups 512 bytes apart.
__device__ __forceinline__ uint64_t sdesc_k64b(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused when swizzled)
  d |= (uint64_t)(512u >> 4) << 32;          // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)4 << 61;                    // swizzle mode: 64 B
  return d;
}

// Instruction descriptor, kind::f16: D fp32, A and B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------- vector add

// Elementwise tasks over [lo, hi), by threads tid = 0 .. nthr-1 (a CTA's
// share of one tile): float4 streaming loads (evict-first), 4 in flight per
// thread, scalar head/tail when the operands are not 16-byte aligned there.
//   ELEM_ADD: c[i] = a[i] + b[i]                     (Table 2, VecAdd)
//   ELEM_MUL: c[i] = (...((a[i] * b[i]) * b[i])...) * b[i], `iters` products
//             (Table 2, VecMul: 15 iterations), each rounded to nearest
enum : int { kElemAdd = 0, kElemMul = 1 };

template <int OP>
__device__ __forceinline__ float elem_op(float x, float y, int iters) {
  if (OP == kElemAdd) return __fadd_rn(x, y);
  float z = x;
  for (int i = 0; i < iters; ++i) z = __fmul_rn(z, y);
  return z;
}

template <int OP>
__device__ __forceinline__ void elementwise_range(const float* __restrict__ a, const float* __restrict__ b,
                                                  float* __restrict__ c, int64_t lo, int64_t hi, int tid, int nthr,
                                                  int iters) {
  const bool vec = ((reinterpret_cast<uintptr_t>(a + lo) | reinterpret_cast<uintptr_t>(b + lo) |
                     reinterpret_cast<uintptr_t>(c + lo)) &
                    15) == 0;
  int64_t done = lo;
  if (vec) {
    const int64_t nv = (hi - lo) >> 2;
    const float4* a4 = reinterpret_cast<const float4*>(a + lo);
    const float4* b4 = reinterpret_cast<const float4*>(b + lo);
    float4* c4 = reinterpret_cast<float4*>(c + lo);
    constexpr int U = 4;
    int64_t i = tid;
    for (; i + (int64_t)(U - 1) * nthr < nv; i += (int64_t)U * nthr) {
      float4 x[U], y[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        x[u] = __ldcs(a4 + i + u * nthr);
        y[u] = __ldcs(b4 + i + u * nthr);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        float4 z;
        z.x = elem_op<OP>(x[u].x, y[u].x, iters);
        z.y = elem_op<OP>(x[u].y, y[u].y, iters);
        z.z = elem_op<OP>(x[u].z, y[u].z, iters);
        z.w = elem_op<OP>(x[u].w, y[u].w, iters);
        __stcs(c4 + i + u * nthr, z);
      }
    }
    for (; i < nv; i += nthr) {
      const float4 x = __ldcs(a4 + i), y = __ldcs(b4 + i);
      float4 z;
      z.x = elem_op<OP>(x.x, y.x, iters);
      z.y = elem_op<OP>(x.y, y.y, iters);
      z.z = elem_op<OP>(x.z, y.z, iters);
      z.w = elem_op<OP>(x.w, y.w, iters);
      __stcs(c4 + i, z);
    }
    done = lo + (nv << 2);
  }
  for (int64_t i = done + tid; i < hi; i += nthr) c[i] = elem_op<OP>(a[i], b[i], iters);
}

__device__ __forceinline__ void vadd_range(const float* __restrict__ a, const float* __restrict__ b,
                                           float* __restrict__ c, int64_t lo, int64_t hi, int tid, int nthr) {
  elementwise_range<kElemAdd>(a, b, c, lo, hi, tid, nthr, 0);
}
__device__ __forceinline__ void vmul_range(const float* __restrict__ a, const float* __restrict__ b,
                                           float* __restrict__ c, int64_t lo, int64_t hi, int tid, int nthr,
                                           int iters) {
  elementwise_range<kElemMul>(a, b, c, lo, hi, tid, nthr, iters);
}

// ---------------------------------------------------------------- FMA SGEMM

struct FmaSmem {
  float As[2][kFmaBK][kFmaTile + 4];  // k-major copy of the A panel
  float Bs[2][kFmaBK][kFmaTile + 4];
};

// One 128 x 128 tile (tm, tn) of C = A B in binary32 FMA, by 256 threads.
// Every output accumulates k = 0, 1, ..., K-1 in order in one register.
__device__ __forceinline__ void fma_tile(const float* __restrict__ A, const float* __restrict__ B,
                                         float* __restrict__ C, int m, int n, int k, int tm, int tn,
                                         FmaSmem* s) {
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int row0 = tm * kFmaTile, col0 = tn * kFmaTile;
  const bool vec = ((k & 3) == 0) && ((n & 3) == 0) &&
                   ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) == 0;
  const int la_r = tid >> 1, la_k = (tid & 1) * 8;    // A panel: row, k offset
  const int lb_k = tid >> 4, lb_c = (tid & 15) * 8;  // B panel: k, column offset
  float ra[8], rb[8];

  auto load = [&](int kt) {
    const int kb = kt * kFmaBK;
    const int r = row0 + la_r, kk = kb + la_k;
    const int bk = kb + lb_k, c = col0 + lb_c;
    if (vec) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < m && kk + 4 * h < k) v = *reinterpret_cast<const float4*>(A + (int64_t)r * k + kk + 4 * h);
        ra[4 * h + 0] = v.x; ra[4 * h + 1] = v.y; ra[4 * h + 2] = v.z; ra[4 * h + 3] = v.w;
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (bk < k && c + 4 * h < n) w = *reinterpret_cast<const float4*>(B + (int64_t)bk * n + c + 4 * h);
        rb[4 * h + 0] = w.x; rb[4 * h + 1] = w.y; rb[4 * h + 2] = w.z; rb[4 * h + 3] = w.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        ra[i] = (r < m && kk + i < k) ? A[(int64_t)r * k + kk + i] : 0.f;
        rb[i] = (bk < k && c + i < n) ? B[(int64_t)bk * n + c + i] : 0.f;
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < 8; ++i) s->As[buf][la_k + i][la_r] = ra[i];
    *reinterpret_cast<float4*>(&s->Bs[buf][lb_k][lb_c]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    *reinterpret_cast<float4*>(&s->Bs[buf][lb_k][lb_c + 4]) = make_float4(rb[4], rb[5], rb[6], rb[7]);
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  const int nkt = (k + kFmaBK - 1) / kFmaBK;
  load(0);
  store(0);
  __syncthreads();
  for (int kt = 0; kt < nkt; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nkt) load(kt + 1);
#pragma unroll
    for (int kk = 0; kk < kFmaBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&s->As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&s->As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&s->Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&s->Bs[buf][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = __fmaf_rn(av[i], bv[j], acc[i][j]);
    }
    if (kt + 1 < nkt) store(buf ^ 1);
    __syncthreads();
  }

  const bool cvec = ((n & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (r >= m) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = col0 + h * 64 + tx * 4;
      float* dst = C + (int64_t)r * n + c;
      if (cvec && c + 3 < n) {
        *reinterpret_cast<float4*>(dst) =
            make_float4(acc[i][4 * h + 0], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (c + j < n) dst[j] = acc[i][4 * h + j];
      }
    }
  }
}

// ---------------------------------------------------------------- split3 pre-pass

// x = hi + lo + r with hi = bf16(x), lo = bf16(x - hi); x - hi is exact in binary32.
__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(__fsub_rn(v[2 * i], hf.x), __fsub_rn(v[2 * i + 1], hf.y));
    h[i] = *reinterpret_cast<const uint32_t*>(&hb);
    l[i] = *reinterpret_cast<const uint32_t*>(&lb);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Rows [r0, r0 + rows) of A (m x k, row-major) into the hi plane
// (planes + row * kp) and the lo plane (+ m * kp). Columns k .. kp-1 get 0.
// Threads tid = 0 .. nthr-1 take groups of 8 elements; each keeps
// kSplitUnroll groups in flight, so that a CTA has ~32 KB of loads
// outstanding (the pass is bound by memory latency otherwise).
constexpr int kSplitUnroll = 4;

__device__ __forceinline__ void split_a_tile(const float* __restrict__ A, __nv_bfloat16* __restrict__ planes,
                                             int m, int k, int kp, int r0, int rows, int tid, int nthr) {
  const int groups = kp >> 3;
  rows = min(rows, m - r0);
  const bool vec = ((k & 3) == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
  const int64_t total = (int64_t)rows * groups;
  for (int64_t gb = 0; gb < total; gb += (int64_t)nthr * kSplitUnroll) {
    float v[kSplitUnroll][8];
#pragma unroll
    for (int u = 0; u < kSplitUnroll; ++u) {
      const int64_t g = gb + tid + (int64_t)u * nthr;
      if (g >= total) continue;
      const int r = r0 + (int)(g / groups);
      const int kk = (int)(g % groups) * 8;
      const float* src = A + (int64_t)r * k + kk;
      if (vec && kk + 8 <= k) {
        const float4 x0 = __ldcs(reinterpret_cast<const float4*>(src));
        const float4 x1 = __ldcs(reinterpret_cast<const float4*>(src + 4));
        v[u][0] = x0.x; v[u][1] = x0.y; v[u][2] = x0.z; v[u][3] = x0.w;
        v[u][4] = x1.x; v[u][5] = x1.y; v[u][6] = x1.z; v[u][7] = x1.w;
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) v[u][i] = (kk + i < k) ? src[i] : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < kSplitUnroll; ++u) {
      const int64_t g = gb + tid + (int64_t)u * nthr;
      if (g >= total) continue;
      const int r = r0 + (int)(g / groups);
      const int kk = (int)(g % groups) * 8;
      uint4 hi, lo;
      split8(v[u], hi, lo);
      st_cg_v4(planes + (int64_t)r * kp + kk, hi);
      st_cg_v4(planes + (int64_t)m * kp + (int64_t)r * kp + kk, lo);
    }
  }
}

// Columns [c0, c0 + cols) of B (k x n, row-major) into rows of the
// transposed planes: hi at planes + col * kp, lo at + n * kp. Work items are
// (32 columns, 8 rows of B); warp w of the nthr/32 warps takes items w, w +
// nwarps, ... so every load instruction reads 32 consecutive floats of one
// row of B, and each lane keeps kSplitUnroll items (32 loads) in flight.
__device__ __forceinline__ void split_b_tile(const float* __restrict__ B, __nv_bfloat16* __restrict__ planes,
                                             int64_t n, int k, int kp, int64_t c0, int cols, int tid, int nthr) {
  cols = (int)min((int64_t)cols, n - c0);
  const int lane = tid & 31, w = tid >> 5, nw = nthr >> 5;
  const int cgroups = (cols + 31) >> 5, kgroups = kp >> 3;
  const int items = cgroups * kgroups;
  for (int ib = w; ib < items; ib += nw * kSplitUnroll) {
    float v[kSplitUnroll][8];
#pragma unroll
    for (int u = 0; u < kSplitUnroll; ++u) {
      const int item = ib + u * nw;
      const int cg = item % cgroups, kg = item / cgroups;
      const int c = cg * 32 + lane;
      const int kk = kg * 8;
      const bool live = item < items && c < cols;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        v[u][i] = (live && kk + i < k) ? __ldcs(B + (int64_t)(kk + i) * n + c0 + c) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kSplitUnroll; ++u) {
      const int item = ib + u * nw;
      const int cg = item % cgroups, kg = item / cgroups;
      const int c = cg * 32 + lane;
      if (item >= items || c >= cols) continue;
      const int64_t col = c0 + c;
      const int kk = kg * 8;
      uint4 hi, lo;
      split8(v[u], hi, lo);
      st_cg_v4(planes + col * kp + kk, hi);
      st_cg_v4(planes + n * kp + col * kp + kk, lo);
    }
  }
}

// ---------------------------------------------------------------- tcgen05 GEMM tile

// Shared state of the tensor-core pipeline (static shared memory).
struct TcShared {
  uint64_t full[kTcStages];   // TMA -> MMA: stage filled
  uint64_t empty[kTcStages];  // MMA -> TMA: stage consumed
  uint64_t accum;             // MMA -> epilogue: accumulator complete
  uint32_t tmem_base;
  uint32_t pad;
};

constexpr uint32_t kTcAOff = 0;                                  // A hi  [kTcM][kTcBK]
constexpr uint32_t kTcAlOff = kTcM * kTcBK * 2;                  // A lo
constexpr uint32_t kTcBOff = 2 * kTcM * kTcBK * 2;               // B^T hi [kTcN][kTcBK]
constexpr uint32_t kTcBlOff = kTcBOff + kTcN * kTcBK * 2;        // B^T lo
static_assert(kTcBlOff + kTcN * kTcBK * 2 == kTcStageBytes, "stage layout");
constexpr uint32_t kTcIdesc = idesc_bf16_f32(kTcM, kTcN);
constexpr uint32_t kTmemCols = kTcN;  // one fp32 accumulator of kTcM lanes x kTcN columns

__device__ __forceinline__ void tc_init(TcShared* ts) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&ts->full[s], 1);
      mbar_init(&ts->empty[s], 1);
    }
    mbar_init(&ts->accum, 1);
    mbar_fence_init();
  }
  if ((threadIdx.x >> 5) == 1) tmem_alloc(&ts->tmem_base, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ __forceinline__ void tc_teardown(TcShared* ts) {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if ((threadIdx.x >> 5) == 1) tmem_dealloc(ts->tmem_base, kTmemCols);
}

// One kTcM x kTcN tile (tm, tn) of C = AhBh + AhBl + AlBh from the bf16 planes
// described by tmA / tmB. Called by all 256 threads of the CTA: warp 0 issues
// TMA, warp 1 issues MMA, warps 4..7 drain TMEM into C. `it` counts pipeline
// stages used so far and `tile_no` tiles so far (identical in every thread).
// split_done / nsplit: the producer first waits until the split pre-pass of
// this task has finished (NULL when the planes are already complete).
// tmap_global: the tensor maps live in global memory written by generic
// stores (the scheduler's task table) and need a proxy acquire fence.
// On a wait that runs out, sets *cta_abort; the CTA must stop afterwards.
__device__ __forceinline__ void tc_tile(const CUtensorMap* tmA, const CUtensorMap* tmB, float* __restrict__ C,
                                        int m, int64_t n, int k, int tm, int tn, uint8_t* stages, TcShared* ts,
                                        uint32_t& it, uint32_t& tile_no, uint64_t timeout_ns,
                                        const uint32_t* split_done, uint32_t nsplit,
                                        volatile uint32_t* cta_abort, uint32_t* fail_where, bool tmap_global,
                                        uint64_t* wait_acc = nullptr) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (k + kTcBK - 1) / kTcBK;
  if (warp == 0) {
    if (lane == 0) {
      bool ok = true;
      if (split_done != nullptr) {
        const uint64_t t0 = globaltimer();
        const uint64_t deadline = t0 + timeout_ns;
        while (ld_acquire_gpu(split_done) < nsplit) {
          if (*cta_abort || globaltimer() > deadline) {
            ok = false;
            *fail_where = kWhereSplitWait;
            break;
          }
          __nanosleep(256);
        }
        if (wait_acc) *wait_acc += globaltimer() - t0;
      }
      fence_proxy_async_global();
      if (tmap_global) {
        fence_tensormap_acquire(tmA);
        fence_tensormap_acquire(tmB);
      }
      for (int kb = 0; ok && kb < nkb; ++kb) {
        const uint32_t q = it + kb, s = q % kTcStages, ph = (q / kTcStages) & 1;
        if (!mbar_wait(&ts->empty[s], ph ^ 1, timeout_ns, cta_abort)) {
          ok = false;
          *fail_where = kWhereEmptyBarrier;
          break;
        }
        uint8_t* st = stages + s * kTcStageBytes;
        mbar_expect_tx(&ts->full[s], kTcStageBytes);
        const int kc = kb * kTcBK;
        tma_load_3d(st + kTcAOff, tmA, kc, tm * kTcM, 0, &ts->full[s]);
        tma_load_3d(st + kTcAlOff, tmA, kc, tm * kTcM, 1, &ts->full[s]);
        tma_load_3d(st + kTcBOff, tmB, kc, tn * kTcN, 0, &ts->full[s]);
        tma_load_3d(st + kTcBlOff, tmB, kc, tn * kTcN, 1, &ts->full[s]);
      }
      if (!ok) *cta_abort = 1;
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      const uint32_t tmem = ts->tmem_base;
      for (int kb = 0; kb < nkb; ++kb) {
        const uint32_t q = it + kb, s = q % kTcStages, ph = (q / kTcStages) & 1;
        if (!mbar_wait(&ts->full[s], ph, timeout_ns, cta_abort)) {
          ok = false;
          *fail_where = kWhereFullBarrier;
          break;
        }
        tc_fence_after();
        const uint32_t base = smem_u32(stages + s * kTcStageBytes);
        const uint64_t dAh = sdesc_k64b(base + kTcAOff), dAl = sdesc_k64b(base + kTcAlOff);
        const uint64_t dBh = sdesc_k64b(base + kTcBOff), dBl = sdesc_k64b(base + kTcBlOff);
#pragma unroll
        for (int kk = 0; kk < kTcBK / 16; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K
          umma_bf16(tmem, dAl + adv, dBh + adv, kTcIdesc, (kb | kk) ? 1u : 0u);
          umma_bf16(tmem, dAh + adv, dBl + adv, kTcIdesc, 1u);
          umma_bf16(tmem, dAh + adv, dBh + adv, kTcIdesc, 1u);
        }
        umma_commit(&ts->empty[s]);
      }
      if (ok) umma_commit(&ts->accum);
      else *cta_abort = 1;
    }
    __syncwarp();
  } else if (warp >= 4) {
    const int q = warp - 4;
    if (!mbar_wait(&ts->accum, tile_no & 1, timeout_ns, cta_abort)) {
      if (lane == 0) {
        *fail_where = kWhereAccumBarrier;
        *cta_abort = 1;
      }
    } else {
      tc_fence_after();
      // TMEM gives each thread one row; a 32 x 32 block goes through a
      // warp-private shared-memory tile (row pitch 33 words: no bank
      // conflicts either way) so that every store of the warp writes 32
      // consecutive floats of one row of C. The pipeline stages are free:
      // every MMA of this tile has completed.
      float* stage = reinterpret_cast<float*>(stages) + q * (32 * 33);
      const int row0 = tm * kTcM + q * 32;
#pragma unroll 1
      for (int ch = 0; ch < kTcN / 32; ++ch) {
        uint32_t r[32];
        tmem_ld_32x32b_x32(ts->tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(ch * 32), r);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(r[j]);
        __syncwarp();
        const int64_t c = (int64_t)tn * kTcN + ch * 32 + lane;
        if (c < n) {
          const int rows = min(32, m - row0);
#pragma unroll 4
          for (int i = 0; i < rows; ++i) C[(int64_t)(row0 + i) * n + c] = stage[i * 33 + lane];
        }
        __syncwarp();
      }
    }
    tc_fence_before();
  }
  it += (uint32_t)nkb;
  tile_no += 1;
}

}  // namespace gvm
