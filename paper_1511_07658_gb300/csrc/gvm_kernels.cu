// The task kernels on their own: gvm_vadd_f32 and gvm_sgemm_f32 run one
// task's kernel on caller-given device buffers without the manager. They use
// the same tile functions as the scheduler, so a task computed here and the
// same task computed by the manager agree bit for bit.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "gvm.h"
#include "gvm_device.cuh"
#include "gvm_fused.cuh"
#include "gvm_wide.cuh"
#include "gvm_runtime.h"

namespace gvm {

// Last error status of a standalone kernel (0 = ok); see gvm_kernel_status.
__device__ uint32_t g_kernel_status;

__global__ void __launch_bounds__(kThreads) vadd_kernel(const float* a, const float* b, float* c, int64_t n,
                                                        int64_t chunk) {
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  if (lo >= n) return;
  vadd_range(a, b, c, lo, min(n, lo + chunk), threadIdx.x, kThreads);
}

__global__ void __launch_bounds__(kThreads) vmul_kernel(const float* a, const float* b, float* c, int64_t n,
                                                        int64_t chunk, int iters) {
  const int64_t lo = (int64_t)blockIdx.x * chunk;
  if (lo >= n) return;
  vmul_range(a, b, c, lo, min(n, lo + chunk), threadIdx.x, kThreads, iters);
}

__global__ void __launch_bounds__(kThreads, 2) fma_sgemm_kernel(const float* A, const float* B, float* C, int m,
                                                                 int n, int k) {
  extern __shared__ uint8_t dyn_smem[];
  fma_tile(A, B, C, m, n, k, blockIdx.y, blockIdx.x, reinterpret_cast<FmaSmem*>(dyn_smem));
}

// Standalone split pass: finer tiles than the scheduler's so that one task
// alone spreads over more SMs.
constexpr int kSplitRowsAlone = 32;

__global__ void __launch_bounds__(kThreads) split_kernel(const float* A, const float* B, __nv_bfloat16* pa,
                                                         __nv_bfloat16* pb, int m, int n, int k, int kp) {
  const int tiles_a = (m + kSplitRowsAlone - 1) / kSplitRowsAlone;
  const int t = blockIdx.x;
  if (t < tiles_a) {
    split_a_tile(A, pa, m, k, kp, t * kSplitRowsAlone, kSplitRowsAlone, threadIdx.x, kThreads);
  } else {
    split_b_tile(B, pb, n, k, kp, (int64_t)(t - tiles_a) * kSplitRowsAlone, kSplitRowsAlone, threadIdx.x,
                 kThreads);
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    tc_sgemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, float* C,
                    int m, int n, int k, uint64_t timeout_ns) {
  __shared__ TcShared ts;
  __shared__ uint32_t abort_flag, fail_where;
  extern __shared__ uint8_t dyn_smem[];
  uint8_t* big = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023));
  if (threadIdx.x == 0) {
    abort_flag = 0;
    fail_where = 0;
  }
  tc_init(&ts);
  uint32_t it = 0, tile_no = 0;
  tc_tile(&tmA, &tmB, C, m, n, k, blockIdx.y, blockIdx.x, big, &ts, it, tile_no, timeout_ns, nullptr, 0,
          &abort_flag, &fail_where, false);
  tc_teardown(&ts);
  if (threadIdx.x == 0 && abort_flag) atomicExch(&g_kernel_status, kStatusTimeout | (fail_where << 8));
}

// Fused split3 GEMM over all tiles of one product: a persistent grid, CTA i
// takes tiles i, i + grid, ... (row-major over the tile grid). Every role
// walks the same tile sequence; the control warp has nothing to do here.
__global__ void __launch_bounds__(kFzThreads, 1)
    fz_sgemm_kernel(const float* A, const float* B, float* C, int m, int n, int k, uint64_t timeout_ns) {
  __shared__ FzShared fs;
  __shared__ uint32_t abort_flag, fail_where;
  extern __shared__ uint8_t dyn_smem[];
  uint8_t* big = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023));
  if (threadIdx.x == 0) {
    abort_flag = 0;
    fail_where = 0;
  }
  fz_init(&fs);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = (n + kTcN - 1) / kTcN;
  const int ntiles = ((m + kTcM - 1) / kTcM) * tiles_n;
  const uint32_t nkb = (uint32_t)((k + kTcBK - 1) / kTcBK);
  uint32_t it = 0, tile_no = 0;
  if (warp < kFzConvWarps) {
    FzTile prev{};
    bool have_prev = false, ok = true;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
      const FzTile t{A, B, C, n, m, k, tile / tiles_n, tile % tiles_n};
      ok = fz_convert<false>(t, big, &fs, it, timeout_ns, &abort_flag, &fail_where, nullptr);
      if (ok && have_prev) ok = fz_epilogue(prev, &fs, tile_no - 1, timeout_ns, &abort_flag, &fail_where);
      prev = t;
      have_prev = true;
      it += nkb;
      ++tile_no;
    }
    if (ok && have_prev) fz_epilogue(prev, &fs, tile_no - 1, timeout_ns, &abort_flag, &fail_where);
  } else if (warp == kFzMmaWarp) {
    if (lane == 0) {
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const FzTile t{A, B, C, n, m, k, tile / tiles_n, tile % tiles_n};
        if (!fz_mma(t, big, &fs, it, tile_no, timeout_ns, &abort_flag, &fail_where, nullptr)) break;
        it += nkb;
        ++tile_no;
      }
    }
    __syncwarp();
  }
  fz_teardown(&fs);
  if (threadIdx.x == 0 && abort_flag) atomicExch(&g_kernel_status, kStatusTimeout | (fail_where << 8));
}

// Wide form: 256 x 256 tiles, the same static tile order; a tile's
// accumulator is drained by the converters right after their first k-step of
// the next tile (one accumulator fills TMEM).
__global__ void __launch_bounds__(kFzThreads, 1)
    wd_sgemm_kernel(const __grid_constant__ CUtensorMap tmA, int a_tma, const float* A, const float* B, float* C,
                    int m, int n, int k, uint64_t timeout_ns) {
  __shared__ WdShared ws;
  __shared__ uint32_t abort_flag, fail_where;
  extern __shared__ uint8_t dyn_smem[];
  uint8_t* big = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023));
  if (threadIdx.x == 0) {
    abort_flag = 0;
    fail_where = 0;
  }
  wd_init(&ws);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = (n + kWdN - 1) / kWdN;
  const int ntiles = ((m + kWdM - 1) / kWdM) * tiles_n;
  const uint32_t nkb = (uint32_t)((k + kTcBK - 1) / kTcBK);
  uint32_t it = 0, tile_no = 0;
  if (warp < kFzConvWarps) {
    FzTile prev{};
    bool pending = false, ok = true;
    uint32_t land_n = 0, land_iss = 0;
    auto drain = [&]() -> bool {
      if (!pending) return true;
      pending = false;
      return wd_epilogue(prev, &ws, tile_no - 1, timeout_ns, &abort_flag, &fail_where);
    };
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
      const FzTile t{A, B, C, n, m, k, tile / tiles_n, tile % tiles_n};
      ok = wd_convert(t, big, &ws, it, timeout_ns, &abort_flag, &fail_where, nullptr, drain, land_n, land_iss,
                      a_tma ? &tmA : nullptr);
      if (ok) ok = drain();  // this group had no k-step of the tile
      prev = t;
      pending = true;
      it += nkb;
      ++tile_no;
    }
    if (ok) drain();
    wd_land_quiesce(&ws, land_n, land_iss, timeout_ns);
  } else if (warp == kFzMmaWarp) {
    if (lane == 0) {
      for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const FzTile t{A, B, C, n, m, k, tile / tiles_n, tile % tiles_n};
        if (!wd_mma(t, big, &ws, it, tile_no, timeout_ns, &abort_flag, &fail_where, nullptr)) break;
        it += nkb;
        ++tile_no;
      }
    }
    __syncwarp();
  }
  wd_teardown(&ws);
  if (threadIdx.x == 0 && abort_flag) atomicExch(&g_kernel_status, kStatusTimeout | (fail_where << 8));
}

// ---------------------------------------------------------------- driver API

static DriverApi g_api;
static bool g_api_ok = false;
static std::once_flag g_api_once;

const DriverApi* driver_api() {
  std::call_once(g_api_once, [] {
    cudaDriverEntryPointQueryResult q;
    void* f1 = nullptr;
    void* f2 = nullptr;
    void* f3 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &f1, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return;
    if (cudaGetDriverEntryPointByVersion("cuStreamWaitValue32", &f2, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f3, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return;
    void* f4 = nullptr;
    void* f5 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f4, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f5, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return;
    g_api.ctx_get_current = reinterpret_cast<decltype(g_api.ctx_get_current)>(f4);
    g_api.ctx_get_id = reinterpret_cast<decltype(g_api.ctx_get_id)>(f5);
    g_api.write_value32 = reinterpret_cast<decltype(g_api.write_value32)>(f1);
    g_api.wait_value32 = reinterpret_cast<decltype(g_api.wait_value32)>(f2);
    g_api.encode_tiled = reinterpret_cast<decltype(g_api.encode_tiled)>(f3);
    g_api_ok = true;
  });
  return g_api_ok ? &g_api : nullptr;
}

uint64_t current_ctx_id() {
  const DriverApi* api = driver_api();
  if (!api) return 0;
  CUcontext c = nullptr;
  if (api->ctx_get_current(&c) != CUDA_SUCCESS || c == nullptr) return 0;
  unsigned long long id = 0;
  if (api->ctx_get_id(c, &id) != CUDA_SUCCESS) return 0;
  return (uint64_t)id;
}

CUresult encode_split_maps(void* scratch, int32_t m, int64_t n, int32_t k, CUtensorMap* tmA, CUtensorMap* tmB) {
  const DriverApi* api = driver_api();
  if (!api) return CUDA_ERROR_NOT_INITIALIZED;
  const uint64_t kp = split_kp(k);
  uint8_t* pa = static_cast<uint8_t*>(scratch);
  uint8_t* pb = pa + split_a_bytes(m, k);
  const cuuint32_t estr[3] = {1, 1, 1};
  {
    const cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)m, 2};
    const cuuint64_t strides[2] = {kp * 2, (cuuint64_t)m * kp * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kTcBK, (cuuint32_t)kTcM, 1};
    CUresult r = api->encode_tiled(tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, pa, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return r;
  }
  {
    const cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)n, 2};
    const cuuint64_t strides[2] = {kp * 2, (cuuint64_t)n * kp * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kTcBK, (cuuint32_t)kTcN, 1};
    return api->encode_tiled(tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, pb, dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
}

CUresult encode_wide_a_map(const float* A, int32_t m, int32_t k, CUtensorMap* tm) {
  // A box of 256 rows x 32 binary32 values, written densely (128-byte rows)
  // into shared memory; rows beyond m and columns beyond k read as zero. The
  // row pitch must be a multiple of 16 bytes and A 16-byte aligned.
  if ((k % 4) != 0 || (reinterpret_cast<uintptr_t>(A) & 15) != 0) return CUDA_ERROR_INVALID_VALUE;
  const DriverApi* api = driver_api();
  if (!api) return CUDA_ERROR_NOT_INITIALIZED;
  const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)m};
  const cuuint64_t strides[1] = {(cuuint64_t)k * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)kWdM};
  const cuuint32_t estr[2] = {1, 1};
  return api->encode_tiled(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

CUresult encode_tma_maps(const float* A, const float* B, int32_t m, int64_t n, int32_t k, CUtensorMap* tmA,
                         CUtensorMap* tmB, int* b3) {
  // A: boxes of 128 rows x 32 values; B: boxes of 32 rows (k) x 32 columns.
  // Each lands as 128-byte rows with the 128-byte swizzle (16-byte chunk j of
  // row r at chunk j ^ (r % 8)); elements beyond the matrix read as zero.
  if ((k % 4) != 0 || (n % 4) != 0 || ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) != 0)
    return CUDA_ERROR_INVALID_VALUE;
  const DriverApi* api = driver_api();
  if (!api) return CUDA_ERROR_NOT_INITIALIZED;
  const cuuint32_t estr[2] = {1, 1};
  {
    const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)m};
    const cuuint64_t strides[1] = {(cuuint64_t)k * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)kTcM};
    CUresult r = api->encode_tiled(tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box,
                                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return r;
  }
  *b3 = 0;
  if (n % 32 == 0) {
    // B as (column within its 32-column slab, k, slab): a box of {32, kTcBK,
    // 8} lands the eight slabs of a tile's k-step one after another, each as
    // kTcBK rows of 128 bytes: the layout of eight 2D boxes, in one copy.
    const cuuint64_t dims3[3] = {32, (cuuint64_t)k, (cuuint64_t)(n / 32)};
    const cuuint64_t strides3[2] = {(cuuint64_t)n * 4, 128};
    const cuuint32_t box3[3] = {32, (cuuint32_t)kTcBK, (cuuint32_t)(kTcN / 32)};
    const cuuint32_t estr3[3] = {1, 1, 1};
    if (api->encode_tiled(tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(B), dims3, strides3, box3,
                          estr3, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
      *b3 = 1;
      return CUDA_SUCCESS;
    }
  }
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)k};
  const cuuint64_t strides[1] = {(cuuint64_t)n * 4};
  const cuuint32_t box[2] = {32, (cuuint32_t)kTcBK};
  return api->encode_tiled(tmB, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(B), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

constexpr uint64_t kStandaloneTimeoutNs = 10ull * 1000 * 1000 * 1000;

static int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  }
  return sms;
}

}  // namespace gvm

using namespace gvm;

extern "C" int gvm_vadd_f32(const float* a, const float* b, float* c, int64_t n, void* stream) {
  if (n < 0) return GVM_EINVAL;
  if (n == 0) return GVM_OK;
  if (!a || !b || !c) return GVM_EINVAL;
  const int sms = sm_count();
  if (sms <= 0) return GVM_ENODEV;
  int64_t chunk = (n + (int64_t)sms * 4 - 1) / ((int64_t)sms * 4);
  chunk = (chunk + 1023) / 1024 * 1024;
  if (chunk < kVaddTileMin) chunk = kVaddTileMin;
  const int64_t grid = (n + chunk - 1) / chunk;
  vadd_kernel<<<(unsigned)grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(a, b, c, n, chunk);
  return cudaGetLastError() == cudaSuccess ? GVM_OK : GVM_EDEVICE;
}

extern "C" int gvm_vmul_f32(const float* a, const float* b, float* c, int64_t n, int32_t iters, void* stream) {
  if (n < 0 || iters < 1 || iters > 1024) return GVM_EINVAL;
  if (n == 0) return GVM_OK;
  if (!a || !b || !c) return GVM_EINVAL;
  const int sms = sm_count();
  if (sms <= 0) return GVM_ENODEV;
  int64_t chunk = (n + (int64_t)sms * 4 - 1) / ((int64_t)sms * 4);
  chunk = (chunk + 1023) / 1024 * 1024;
  if (chunk < kVaddTileMin) chunk = kVaddTileMin;
  const int64_t grid = (n + chunk - 1) / chunk;
  vmul_kernel<<<(unsigned)grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(a, b, c, n, chunk, iters);
  return cudaGetLastError() == cudaSuccess ? GVM_OK : GVM_EDEVICE;
}

extern "C" uint64_t gvm_sgemm_scratch_bytes(int32_t m, int32_t n, int32_t k, int32_t path) {
  if (m <= 0 || n <= 0 || k <= 0) return 0;
  return path == GVM_SGEMM_SPLIT3 ? split_scratch_bytes(m, n, k) : 0;
}

// The large-shared-memory attribute is set on every call, as for the
// scheduler: it belongs to the function in the current context, so a flag
// kept per process would skip it on a second device or after a reset.
template <typename F>
static int allow_smem(F* fn, size_t smem) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess
             ? GVM_OK
             : GVM_EDEVICE;
}

extern "C" int gvm_sgemm_f32(const float* A, const float* B, float* C, int32_t m, int32_t n, int32_t k,
                             int32_t path, void* scratch, uint64_t scratch_bytes, void* stream) {
  if (m <= 0 || n <= 0 || k <= 0 || m > 65536 || n > 65536 || k > 65536) return GVM_EINVAL;
  if (!A || !B || !C) return GVM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (path == GVM_SGEMM_FMA) {
    const size_t smem = sizeof(FmaSmem);
    if (allow_smem(fma_sgemm_kernel, smem) != GVM_OK) return GVM_EDEVICE;
    dim3 grid((n + kFmaTile - 1) / kFmaTile, (m + kFmaTile - 1) / kFmaTile);
    fma_sgemm_kernel<<<grid, kThreads, smem, s>>>(A, B, C, m, n, k);
    return cudaGetLastError() == cudaSuccess ? GVM_OK : GVM_EDEVICE;
  }
  if (path == GVM_SGEMM_SPLIT3_FUSED) {
    const size_t smem = (size_t)kTcStages * kTcStageBytes + 1024;
    if (allow_smem(fz_sgemm_kernel, smem) != GVM_OK) return GVM_EDEVICE;
    const int sms = sm_count();
    if (sms <= 0) return GVM_ENODEV;
    const int64_t ntiles = (int64_t)((m + kTcM - 1) / kTcM) * ((n + kTcN - 1) / kTcN);
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    fz_sgemm_kernel<<<grid, kFzThreads, smem, s>>>(A, B, C, m, n, k, kStandaloneTimeoutNs);
    return cudaGetLastError() == cudaSuccess ? GVM_OK : GVM_EDEVICE;
  }
  if (path == GVM_SGEMM_SPLIT3_WIDE) {
    const size_t smem = (size_t)kWdSmemBytes + 1024;
    if (allow_smem(wd_sgemm_kernel, smem) != GVM_OK) return GVM_EDEVICE;
    const int sms = sm_count();
    if (sms <= 0) return GVM_ENODEV;
    const int64_t ntiles = (int64_t)((m + kWdM - 1) / kWdM) * ((n + kWdN - 1) / kWdN);
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    CUtensorMap tmA;
    const int a_tma = encode_wide_a_map(A, m, k, &tmA) == CUDA_SUCCESS ? 1 : 0;
    if (!a_tma) memset(&tmA, 0, sizeof(tmA));
    wd_sgemm_kernel<<<grid, kFzThreads, smem, s>>>(tmA, a_tma, A, B, C, m, n, k, kStandaloneTimeoutNs);
    return cudaGetLastError() == cudaSuccess ? GVM_OK : GVM_EDEVICE;
  }
  if (path != GVM_SGEMM_SPLIT3) return GVM_EINVAL;
  const uint64_t need = split_scratch_bytes(m, n, k);
  if (!scratch || scratch_bytes < need || (reinterpret_cast<uintptr_t>(scratch) & 255)) return GVM_EINVAL;
  CUtensorMap tmA, tmB;
  if (encode_split_maps(scratch, m, n, k, &tmA, &tmB) != CUDA_SUCCESS) return GVM_EDEVICE;
  const int kp = (int)split_kp(k);
  uint8_t* pa = static_cast<uint8_t*>(scratch);
  uint8_t* pb = pa + split_a_bytes(m, k);
  const int nsplit = (m + kSplitRowsAlone - 1) / kSplitRowsAlone + (n + kSplitRowsAlone - 1) / kSplitRowsAlone;
  split_kernel<<<nsplit, kThreads, 0, s>>>(A, B, reinterpret_cast<__nv_bfloat16*>(pa),
                                           reinterpret_cast<__nv_bfloat16*>(pb), m, n, k, kp);
  if (cudaGetLastError() != cudaSuccess) return GVM_EDEVICE;
  const size_t smem = (size_t)kTcStages * kTcStageBytes + 1024;
  if (allow_smem(tc_sgemm_kernel, smem) != GVM_OK) return GVM_EDEVICE;
  dim3 grid((n + kTcN - 1) / kTcN, (m + kTcM - 1) / kTcM);
  tc_sgemm_kernel<<<grid, kThreads, smem, s>>>(tmA, tmB, C, m, n, k, kStandaloneTimeoutNs);
  return cudaGetLastError() == cudaSuccess ? GVM_OK : GVM_EDEVICE;
}

// Reads and clears the error status of the standalone kernels (0 = ok; else
// low byte = status, next byte = which wait). Synchronous.
extern "C" int gvm_kernel_status(uint32_t* out) {
  if (!out) return GVM_EINVAL;
  uint32_t v = 0;
  if (cudaMemcpyFromSymbol(&v, g_kernel_status, sizeof(v)) != cudaSuccess) return GVM_EDEVICE;
  const uint32_t zero = 0;
  if (cudaMemcpyToSymbol(g_kernel_status, &zero, sizeof(zero)) != cudaSuccess) return GVM_EDEVICE;
  *out = v;
  return GVM_OK;
}
