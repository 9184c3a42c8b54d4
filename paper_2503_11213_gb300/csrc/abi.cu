// Library-wide C ABI helpers: status strings, version, last CUDA error, the
// device status query, the poll limit of the bounded completion waits and
// the FP32 throughput probe.
#include <atomic>

#include "common.cuh"

namespace sd {
namespace {
thread_local int t_last_cuda_error = 0;
// -1: every kernel uses its own default poll limit
std::atomic<long long> g_wait_limit{-1};
}  // namespace
void set_cuda_error(cudaError_t e) { t_last_cuda_error = (int)e; }

uint32_t wait_limit(uint32_t dflt) {
  const long long v = g_wait_limit.load(std::memory_order_relaxed);
  return v < 0 ? dflt : (uint32_t)v;
}

// 16 independent FMA chains per thread, unrolled: the loop carries 32 flops
// per iteration and chain, nothing else issues in steady state.
__global__ void __launch_bounds__(256) fp32_peak_kernel(float* __restrict__ sink, int iters,
                                                        float a, float b) {
  float x[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = (float)(threadIdx.x & 7) * 1e-3f + (float)k;
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 16; ++k) s += x[k];
  // never true for the arguments the host passes; keeps the chains alive
  if (s == -1.f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace sd

#ifdef SD_CHECKED
namespace sd {
sd_status check_take_lens_trace(int32_t*);
sd_status check_take_render(int32_t*);
sd_status check_take_render_bwd(int32_t*);
sd_status check_take_render_map(int32_t*);
sd_status check_take_render_tc(int32_t*);
sd_status check_take_mlp(int32_t*);
}  // namespace sd
#endif

extern "C" {

const char* sd_status_string(sd_status s) {
  switch (s) {
    case SD_OK: return "ok";
    case SD_ERR_ARG: return "invalid argument";
    case SD_ERR_LENS: return "invalid lens prescription";
    case SD_ERR_UNSUPPORTED: return "unsupported configuration";
    case SD_ERR_CUDA: return "CUDA runtime error";
    case SD_ERR_CAPACITY: return "library table full";
    case SD_ERR_TIMEOUT: return "a bounded device wait gave up";
    default: return "unknown status";
  }
}

int sd_last_cuda_error(void) { return sd::t_last_cuda_error; }

int sd_version(void) { return 200; }

sd_status sd_sync_status(const int32_t* status_word, void* stream) {
  if (!status_word) return SD_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int32_t v = 0;
  SD_CUDA_TRY(cudaMemcpyAsync(&v, status_word, sizeof v, cudaMemcpyDeviceToHost, s));
  SD_CUDA_TRY(cudaStreamSynchronize(s));
  return v != 0 ? SD_ERR_TIMEOUT : SD_OK;
}

sd_status sd_set_wait_limit(long long polls) {
  sd::g_wait_limit.store(polls < 0 ? -1 : (polls > 0xffffffffll ? 0xffffffffll : polls),
                         std::memory_order_relaxed);
  return SD_OK;
}

sd_status sd_check_status(int32_t* site, int32_t* index, int32_t* bound, int64_t* count) {
  if (!site || !count) return SD_ERR_ARG;
#ifdef SD_CHECKED
  SD_CUDA_TRY(cudaDeviceSynchronize());
  sd_status (*const take[])(int32_t*) = {
      sd::check_take_lens_trace, sd::check_take_render, sd::check_take_render_bwd,
      sd::check_take_render_map, sd::check_take_render_tc, sd::check_take_mlp};
  *site = 0;
  *count = 0;
  for (auto f : take) {
    int32_t rec[4];
    const sd_status st = f(rec);
    if (st != SD_OK) return st;
    if (rec[3] == 0) continue;
    if (*site == 0) {
      *site = rec[0];
      if (index) *index = rec[1];
      if (bound) *bound = rec[2];
    }
    *count += rec[3];
  }
  return SD_OK;
#else
  (void)index;
  (void)bound;
  return SD_ERR_UNSUPPORTED;
#endif
}

sd_status sd_dev_fp32_peak(float* sink, int blocks, int iters, void* stream) {
  if (!sink || blocks < 1 || iters < 1) return SD_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  sd::fp32_peak_kernel<<<blocks, 256, 0, s>>>(sink, iters, 0.99990004f, 1.0e-4f);
  return sd::launch_status();
}

}  // extern "C"
