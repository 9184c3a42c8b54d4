// Tensor-core (tcgen05) building blocks of the BF16 render, and a device
// check of them: one CTA computes D = A_u B^T on the tensor core, where A_u
// is a 128-row window (starting at row u) of a K-major BF16 matrix in shared
// memory, B is K-major, K = 32 in two MMAs, and D lives in tensor memory.
// The window start is a plain shift of the descriptor's start address by u
// rows (16 bytes per row inside the no-swizzle core-matrix layout), which is
// what the render uses to walk a staged image tile row by row.

#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace sd {

constexpr int TCC_ROWS = 136, TCC_K = 32, TCC_M = 128, TCC_N = 16;
constexpr uint32_t TCC_LBO_A = TCC_ROWS * 16, TCC_LBO_B = TCC_N * 16;

__global__ void __launch_bounds__(128) tc_check_kernel(const __nv_bfloat16* __restrict__ A,
                                                       const __nv_bfloat16* __restrict__ B,
                                                       int u, float* __restrict__ D,
                                                       int* __restrict__ status) {
  // K-major core-matrix layouts: element (row, k) of A at byte
  // (k / 8) * LBO_A + row * 16 + (k % 8) * 2, likewise B with its N rows
  __shared__ __align__(128) __nv_bfloat16 As[TCC_ROWS * TCC_K];
  __shared__ __align__(128) __nv_bfloat16 Bs[TCC_N * TCC_K];
  __shared__ uint32_t tslot;
  __shared__ __align__(8) uint64_t bar;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < TCC_ROWS * TCC_K; i += 128) {
    int r = i / TCC_K, k = i - r * TCC_K;
    As[(k >> 3) * (TCC_LBO_A / 2) + r * 8 + (k & 7)] = A[i];
  }
  for (int i = tid; i < TCC_N * TCC_K; i += 128) {
    int n = i / TCC_K, k = i - n * TCC_K;
    Bs[(k >> 3) * (TCC_LBO_B / 2) + n * 8 + (k & 7)] = B[i];
  }
  if (warp == 0) tc::tmem_alloc(&tslot, 32);
  if (tid == 0) tc::mbar_init(&bar, 1);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = tslot;
  if (tid == 0) {
    const uint32_t a0 = tc::smem_u32(As) + (uint32_t)u * 16u, b0 = tc::smem_u32(Bs);
    for (int s = 0; s < TCC_K / 16; ++s) {
      const uint64_t ad = tc::smem_desc(a0 + s * 2 * TCC_LBO_A, TCC_LBO_A, 128);
      const uint64_t bd = tc::smem_desc(b0 + s * 2 * TCC_LBO_B, TCC_LBO_B, 128);
      tc::mma_bf16(taddr, ad, bd, tc::idesc_bf16_f32(TCC_M, TCC_N), s > 0);
    }
    tc::commit(&bar);
  }
  const bool ok = tc::mbar_wait(&bar, 0, 1u << 22);
  tc::fence_after_sync();
  if (!ok && lane == 0) atomicExch(status, 1);
  float v[16];
  tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16), v);
  const int row = 32 * warp + lane;
#pragma unroll
  for (int j = 0; j < 16; ++j) D[row * TCC_N + j] = v[j];
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(taddr, 32);
}

}  // namespace sd

extern "C" sd_status sd_dev_tc_check(const void* a, const void* b, int u, float* d,
                                     int32_t* status, void* stream) {
  using namespace sd;
  if (!a || !b || !d || !status || u < 0 || u > TCC_ROWS - TCC_M) return SD_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  tc_check_kernel<<<1, 128, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(a),
                                    reinterpret_cast<const __nv_bfloat16*>(b), u, d, status);
  return launch_status();
}
