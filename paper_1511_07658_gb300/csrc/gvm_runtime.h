// Internal functions shared by the host runtime translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gvm.h"
#include "gvm_internal.h"

namespace gvm {

enum : int { kPathFma = 0, kPathSplit3 = 1, kPathSplit3Wide = 2, kPathSplit3Tma = 3 };

// Driver entry points, resolved once through the runtime (no link-time libcuda).
struct DriverApi {
  CUresult (*write_value32)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);
  CUresult (*wait_value32)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);
  CUresult (*encode_tiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                           const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                           CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  CUresult (*ctx_get_current)(CUcontext*);
  CUresult (*ctx_get_id)(CUcontext, unsigned long long*);
};
// Returns nullptr if the driver or an entry point is unavailable.
const DriverApi* driver_api();

// Process-unique id of the calling thread's current CUDA context (a context
// created after cudaDeviceReset gets a new id); 0 if there is none.
uint64_t current_ctx_id();

// Encodes the two tensor maps of a split3 task whose bf16 planes start at
// `scratch` (A planes, then B^T planes at scratch + split_a_bytes).
// Returns CUDA_SUCCESS or the driver's error.
CUresult encode_split_maps(void* scratch, int32_t m, int64_t n, int32_t k, CUtensorMap* tmA, CUtensorMap* tmB);

// Tensor map of a row-major binary32 A (m x k) in boxes of 256 rows x 32
// values (out-of-range elements read as zero), for the wide split3 form's
// landing buffers; an error where TMA cannot address A (k not a multiple of
// 4, A not 16-byte aligned).
CUresult encode_wide_a_map(const float* A, int32_t m, int32_t k, CUtensorMap* tm);

// Tensor maps of a row-major binary32 A (m x k) in boxes of 128 rows x 32
// values and of B (k x n): when n is a multiple of 32, a 3D map (columns
// within a 32-column slab, k, slabs) whose one box is a k-step's eight slabs
// (*b3 = 1); otherwise boxes of 32 rows x 32 values (*b3 = 0). For the
// TMA-fed split3 form; an error where TMA cannot address them (pitch not a
// multiple of 16 bytes, base not 16-byte aligned).
CUresult encode_tma_maps(const float* A, const float* B, int32_t m, int64_t n, int32_t k, CUtensorMap* tmA,
                         CUtensorMap* tmB, int* b3);

// Scheduler kernel: occupancy-derived grid for `path`, dynamic smem bytes,
// and an asynchronous launch on `stream`.
cudaError_t scheduler_setup(int path, int* blocks_per_sm, size_t* smem_bytes);
cudaError_t launch_scheduler(int path, const SchedParams& p, int grid, size_t smem, cudaStream_t stream);

// Configuration of a manager, for the library's other host modules.
int ctx_mode(const gvm_ctx* ctx);
int ctx_max_ranks(const gvm_ctx* ctx);
// Counts the gvm_ipc servers using a manager (gvm_shutdown refuses while any is).
void ctx_servers_add(gvm_ctx* ctx, int delta);

}  // namespace gvm
