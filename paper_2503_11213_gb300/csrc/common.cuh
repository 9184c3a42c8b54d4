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
