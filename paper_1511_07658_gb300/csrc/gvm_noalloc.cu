// gvm_sgemm_f32_noalloc: the split3 SGEMM task kernel for callers that
// cannot allocate device memory.
//
// The split3 path needs scratch for the bf16 hi/lo copies of A and B^T. The
// regular entry point (gvm_sgemm_f32) takes that scratch from the caller.
// Some callers have no way to provide it: a plain C program linking this
// library with no device allocator of its own, a framework whose memory pool
// already owns all device memory, or a latency-critical serving loop where
// allocating (and the device-wide synchronisation cudaFree implies) is not
// allowed. For them this entry point uses a fixed scratch array that lives in
// this file's device module instead.
//
// The array is a file-scope __device__ variable of kNoAllocScratchBytes; every
// GPU that loads the library holds it until the process exits. Host code
// cannot use the array's name as a device address (it names a host-side
// stand-in), so the first call on each device asks the runtime for the
// array's device address with cudaGetSymbolAddress while that device is
// current, checks the result, and caches it for that device together with
// the id of the context it belongs to. A call in a different context of the
// same device (after cudaDeviceReset) looks the address up again.
#include <cuda_runtime.h>

#include <mutex>

#include "gvm.h"
#include "gvm_internal.h"
#include "gvm_runtime.h"

namespace {

constexpr uint64_t kNoAllocScratchBytes = 32ull << 20;  // 32 MiB: up to m = n = k = 2048
constexpr int kMaxDevices = 64;

__device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

struct ScratchCache {
  uint64_t ctx_id;
  void* ptr;
};
std::mutex g_mu;
ScratchCache g_cache[kMaxDevices] = {};

// Device address of g_noalloc_scratch in the current device's context (set-up
// on the first call per device and context). Returns nullptr if the runtime
// cannot provide it.
void* scratch_for_current_device(int* err) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *err = GVM_ENODEV;
    return nullptr;
  }
  std::lock_guard<std::mutex> g(g_mu);
  const uint64_t id = gvm::current_ctx_id();
  if (id == 0 || g_cache[dev].ctx_id != id || !g_cache[dev].ptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      *err = GVM_EDEVICE;
      return nullptr;
    }
    // The lookup made the device's primary context current if none was.
    g_cache[dev] = ScratchCache{gvm::current_ctx_id(), p};
  }
  return g_cache[dev].ptr;
}

}  // namespace

extern "C" int gvm_sgemm_f32_noalloc(const float* A, const float* B, float* C, int32_t m, int32_t n, int32_t k,
                                     void* stream) {
  if (m <= 0 || n <= 0 || k <= 0 || !A || !B || !C) return GVM_EINVAL;
  if (gvm::split_scratch_bytes(m, n, k) > kNoAllocScratchBytes) return GVM_ENOMEM;
  int err = GVM_OK;
  void* scratch = scratch_for_current_device(&err);
  if (!scratch) return err;
  // The split pass writes every byte of the planes that the GEMM reads (rows
  // 0..m-1 / 0..n-1, columns 0..kp-1, padding included), so nothing needs
  // clearing between calls.
  return gvm_sgemm_f32(A, B, C, m, n, k, GVM_SGEMM_SPLIT3, scratch, kNoAllocScratchBytes, stream);
}
