// Internal definitions shared by the translation units of libsdirt.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sdirt.h"

namespace sd {

// A named NVTX range around each compute entry point of the C ABI, so that
// a profiler's timeline groups the launches of one call under its name (a
// no-op unless a profiling tool is attached).
struct ApiRange {
  explicit ApiRange(const char* name) { nvtxRangePushA(name); }
  ~ApiRange() { nvtxRangePop(); }
  ApiRange(const ApiRange&) = delete;
  ApiRange& operator=(const ApiRange&) = delete;
};
#define SD_API_RANGE(name) ::sd::ApiRange sd_api_range_(name)

// last CUDA error seen on this host thread
void set_cuda_error(cudaError_t e);

// Poll limit of the tensor-core kernels' bounded completion waits: dflt
// unless sd_set_wait_limit has set a process-wide override.
uint32_t wait_limit(uint32_t dflt);

// ---- checked build -------------------------------------------------------
// Built with -DSD_CHECKED, SD_CHECK(i, n) tests 0 <= i < n before an access
// whose index the kernel computes; a failing test records, in its
// translation unit's device record, the first failing site (SD_TU * 100000
// + line), the index and bound (low 32 bits) and a count, and yields false
// so that the caller skips the access.  In the normal build it is the
// constant true.  sd_check_status reads and clears the records.
#ifndef SD_TU
#define SD_TU 0
#endif
#ifdef SD_CHECKED
namespace {
__device__ int g_check[4];  // one per translation unit: site, index, bound, count
}
__device__ __forceinline__ bool check_index(int site, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  if (atomicCAS(&g_check[0], 0, site) == 0) {
    g_check[1] = (int)i;
    g_check[2] = (int)n;
  }
  atomicAdd(&g_check[3], 1);
  return false;
}
#define SD_CHECK(i, n) ::sd::check_index(SD_TU * 100000 + __LINE__, (long long)(i), (long long)(n))
// Host reader of this translation unit's record (defined once per file by
// SD_CHECK_TU(name)): copies it to rec[4] and clears it.
#define SD_CHECK_TU(name)                                                   \
  namespace sd {                                                            \
  sd_status check_take_##name(int32_t* rec) {                               \
    SD_CUDA_TRY(cudaMemcpyFromSymbol(rec, g_check, sizeof(int) * 4));       \
    const int zero[4] = {0, 0, 0, 0};                                       \
    SD_CUDA_TRY(cudaMemcpyToSymbol(g_check, zero, sizeof zero));            \
    return SD_OK;                                                           \
  }                                                                         \
  }
#else
#define SD_CHECK(i, n) true
#define SD_CHECK_TU(name)
#endif

#define SD_CUDA_TRY(expr)                         \
  do {                                            \
    cudaError_t _e = (expr);                      \
    if (_e != cudaSuccess) {                      \
      ::sd::set_cuda_error(_e);                   \
      return SD_ERR_CUDA;                         \
    }                                             \
  } while (0)

inline sd_status launch_status() {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return SD_ERR_CUDA;
  }
  return SD_OK;
}

// ---- storage conversions -------------------------------------------------
template <class T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

template <class T>
__device__ __forceinline__ T from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

}  // namespace sd
