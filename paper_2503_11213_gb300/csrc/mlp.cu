// DP PSF prediction network (Sec. 3.2, "Pixel-wise DP image rendering
// module"): per pixel, an MLP maps the normalised object point p = (x_n,
// y_n, d_n) through 5 hidden layers of 512 (ReLU) to the 2 ks^2 values of
// (PSF_L, PSF_R); the outputs are clamped at 0 and sum-normalised.
//
// One CTA predicts 128 pixels (the MMA's M) with every layer on the
// 5th-generation tensor cores:
//   * the activations of the 128 pixels live in shared memory as the A
//     operand (BF16, no-swizzle K-major core matrices, 128 KB);
//   * the weights of layers 1..5 are packed on the host into 32 KB chunks of
//     256 output rows x 64 inputs, already in the B operand layout, and one
//     thread streams them in consumption order through a ring of three
//     shared buffers with 1-D bulk copies (the TMA engine), completion
//     counted in bytes on an mbarrier per buffer;
//   * one thread issues the MMAs (M = 128, N = 256, K = 16) into a 512-column
//     FP32 accumulator in tensor memory and commits each buffer back to the
//     copier;
//   * eight warps (two per tensor-memory lane quarter, one per half of the
//     columns) compute layer 0 (3 inputs, CUDA cores), and after every layer
//     read the accumulator, add
//     the bias, apply ReLU and write the next A operand in BF16.  The output
//     layer runs in passes of 512 columns (the accumulator's width): the
//     passes first accumulate each pixel's sum of the clamped outputs, the
//     last one then stores its columns normalised (re-read from tensor
//     memory), and the earlier passes are recomputed to store theirs, so the
//     map is written once, never read back.
// Every wait is bounded; a wait that gives up sets *status and makes the
// other waits of the launch give up too.

#define SD_TU 6  // translation unit id of this file's SD_CHECK sites
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace sd {

constexpr int MH = SD_MLP_HIDDEN;   // hidden width
constexpr int MM = 128;             // pixels per CTA
constexpr int MKC = 32;             // inputs per weight chunk
constexpr int MNC = 256;            // outputs per weight chunk
constexpr int MNB = 5;              // weight ring buffers
constexpr uint32_t MCHUNK = MNC * MKC * 2;        // 16 KB
constexpr int MKPB = MH / MKC;      // chunks per 256-row block of a layer
constexpr uint32_t MA_BYTES = MM * MH * 2;        // 128 KB
constexpr int MEPI = 256;           // epilogue threads: warps 0-7
constexpr int MTHREADS = MEPI + 64;  // + warp 8 MMA issue, warp 9 copies
// per epilogue warp: 32 pixels x 16 outputs staged for coalesced stores
// (rows of 18 floats: conflict-free 8-byte accesses)
constexpr int MSROW = 18;
constexpr uint32_t MSTAGE = (MEPI / 32) * 32 * MSROW * 4;
constexpr uint32_t MWAIT = 1u << 22;

__host__ __device__ inline int mlp_nout(int ks) { return 2 * ks * ks; }
__host__ __device__ inline int mlp_nblk(int ks) { return (mlp_nout(ks) + MNC - 1) / MNC; }
// chunks: 4 hidden layers of (512/256) x (512/64), the output layer nblk x 8
__host__ __device__ inline int mlp_chunks(int ks) { return 4 * 2 * MKPB + mlp_nblk(ks) * MKPB; }
// FP32 tail: layer 0 as [512] x {w_x, w_y, w_d, b0} (one 16-byte load per
// neuron), b1..b4 [512] each, b5 [nblk * 256]
__host__ __device__ inline size_t mlp_tail_floats(int ks) {
  return (size_t)MH * 4 + 4 * (size_t)MH + (size_t)mlp_nblk(ks) * MNC;
}
inline size_t mlp_bytes(int ks) { return (size_t)mlp_chunks(ks) * MCHUNK + 4 * mlp_tail_floats(ks); }

struct MlpParams {
  const unsigned char* blob;
  const float* depth;
  void* out;       // FP32 or BF16 map
  int out_bf16;
  int* status;
  int ks, H, W;
  float d_min, d_scale;  // d_n = (d - d_min) * d_scale - 1
  uint32_t wlim;         // polls of a pipeline wait before it gives up
};

__device__ __forceinline__ bool mwait(uint64_t* bar, uint32_t parity, int* err,
                                      uint32_t limit) {
  if (tc::mbar_wait(bar, parity, limit, err)) return true;
  atomicExch(err, 1);
  return false;
}

// output pass computed by accumulator phase ph >= 4: passes 0..npass-1, then
// 0..npass-2 again
__device__ __forceinline__ int mlp_pass(int ph, int npass) {
  const int j = ph - 4;
  return j < npass ? j : j - npass;
}

__device__ __forceinline__ void named_sync_m(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ uint32_t bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // a in the low half
  return *reinterpret_cast<const uint32_t*>(&h);
}

__global__ void __launch_bounds__(MTHREADS, 1) mlp_kernel(const MlpParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* Abuf = smem;             // element (m, k) at (k/8)*2048 + m*16 + (k%8)*2
  unsigned char* Wbuf = smem + MA_BYTES;  // MNB chunks; (n, k) at (k/8)*4096 + n*16 + (k%8)*2
  float* stage = reinterpret_cast<float*>(Wbuf + (size_t)MNB * MCHUNK);  // MSTAGE bytes
  // s_acc[h]: half h of the accumulator (n block 2q + h of the phase) is
  // complete; s_k0: the second half's MMAs over inputs 0..255 are done (the
  // first half's epilogue may then overwrite those inputs); s_epi[h]: the
  // epilogue of half h has read its accumulator and, for a hidden layer,
  // written inputs 256 h .. 256 h + 255 of the next layer
  __shared__ __align__(8) uint64_t s_full[MNB], s_empty[MNB], s_acc[2], s_k0, s_epi[2], s_done;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ks = P.ks, nout = mlp_nout(ks), nblk = mlp_nblk(ks), nchunk = mlp_chunks(ks);
  const int npass = (nblk + 1) / 2;     // output passes of up to 2 x 256 columns
  const int nphase = 4 + 2 * npass - 1; // accumulator phases (earlier passes twice)
  const long long npix = (long long)P.H * P.W;
  const float* tail = reinterpret_cast<const float*>(P.blob + (size_t)nchunk * MCHUNK);
  const float4* WB0 = reinterpret_cast<const float4*>(tail);  // [512] {w, b0}
  const float* B1 = tail + MH * 4;             // b1, ..., b4 (512 each)
  const float* B5 = B1 + 4 * MH;               // [nblk * 256]

  if (warp == 0) tc::tmem_alloc(&s_tmem, 512);
  if (tid == 0) {
    for (int b = 0; b < MNB; ++b) {
      tc::mbar_init(&s_full[b], 1);
      tc::mbar_init(&s_empty[b], 1);
    }
    for (int h = 0; h < 2; ++h) {
      tc::mbar_init(&s_acc[h], 1);
      tc::mbar_init(&s_epi[h], MEPI / 2);
    }
    tc::mbar_init(&s_k0, 1);
    tc::mbar_init(&s_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;

  if (warp == 9) {
    // ---- weight copier: chunks in consumption order through the ring ------
    if (lane == 0) {
      int last[MNB];  // last copy issued into each buffer
      for (int b = 0; b < MNB; ++b) last[b] = -1;
      int c = 0;                     // copies issued
      bool ok = true;
      for (int ph = 0; ph < nphase && ok; ++ph) {
        const int q = ph < 4 ? 0 : mlp_pass(ph, npass);
        const int nb0 = ph < 4 ? 0 : 2 * q, nb1 = ph < 4 ? 2 : min(nb0 + 2, nblk);
        for (int nb = nb0; nb < nb1 && ok; ++nb)
          for (int kb = 0; kb < MKPB; ++kb, ++c) {
            const int b = c % MNB;
            if (c >= MNB && !mwait(&s_empty[b], (uint32_t)(c / MNB - 1) & 1u, P.status, P.wlim)) {
              ok = false;
              break;
            }
            // blob chunk: hidden layer ph + 1, or the output layer's block nb
            const int chunk = (ph < 4 ? (ph * 2 + nb) * MKPB : (8 + nb) * MKPB) + kb;
            tc::mbar_arrive_expect_tx(&s_full[b], MCHUNK);
            tc::bulk_g2s(Wbuf + (size_t)b * MCHUNK, P.blob + (size_t)chunk * MCHUNK, MCHUNK,
                         &s_full[b]);
            last[b] = c;
          }
      }
      // no copy may still be landing when the CTA ends (after an error the
      // MMA thread may not have consumed them): bounded wait for each
      for (int b = 0; b < MNB; ++b)
        if (last[b] >= 0) tc::mbar_wait(&s_full[b], (uint32_t)(last[b] / MNB) & 1u, MWAIT);
    }
  } else if (warp == 8) {
    // ---- MMA issue --------------------------------------------------------
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(MM, MNC);
      const uint32_t a0 = tc::smem_u32(Abuf), w0 = tc::smem_u32(Wbuf);
      int c = 0;
      bool ok = true;
      // per phase: half 0 over inputs 0..255, (wait for inputs 256..511)
      // half 0 over 256..511, half 1 over 0..255, half 1 over 256..511, so
      // that each half's epilogue runs during the other half's MMAs
      auto run = [&](int ph, int nb, int h, int kb0, int kb1) {
        for (int kb = kb0; kb < kb1 && ok; ++kb, ++c) {
          const int b = c % MNB;
          ok = mwait(&s_full[b], (uint32_t)(c / MNB) & 1u, P.status, P.wlim);
          if (!ok) break;
          tc::fence_after_sync();
#pragma unroll
          for (int s = 0; s < MKC / 16; ++s) {
            const uint64_t ad =
                tc::smem_desc(a0 + (uint32_t)(kb * (MKC / 8) + s * 2) * 2048u, 2048, 128);
            const uint64_t bd =
                tc::smem_desc(w0 + (uint32_t)b * MCHUNK + (uint32_t)s * 2 * 4096u, 4096, 128);
            tc::mma_bf16(tmem + (uint32_t)(h * MNC), ad, bd, idesc, kb > 0 || s > 0);
          }
          tc::commit(&s_empty[b]);
        }
      };
      for (int ph = 0; ph < nphase && ok; ++ph) {
        const int q = ph < 4 ? 0 : mlp_pass(ph, npass);
        const int nb0 = ph < 4 ? 0 : 2 * q;
        const bool two = ph < 4 || nb0 + 1 < nblk;
        ok = ok && mwait(&s_epi[0], (uint32_t)ph & 1u, P.status, P.wlim);
        tc::fence_after_sync();
        run(ph, nb0, 0, 0, MKPB / 2);
        ok = ok && mwait(&s_epi[1], (uint32_t)ph & 1u, P.status, P.wlim);
        tc::fence_after_sync();
        run(ph, nb0, 0, MKPB / 2, MKPB);
        tc::commit(&s_acc[0]);
        if (two) run(ph, nb0 + 1, 1, 0, MKPB / 2);
        tc::commit(&s_k0);
        if (two) run(ph, nb0 + 1, 1, MKPB / 2, MKPB);
        tc::commit(&s_acc[1]);
      }
      // every MMA issued has completed before the tensor memory is freed
      // (also after an error)
      tc::commit(&s_done);
      tc::mbar_wait(&s_done, 0, MWAIT);
    }
  } else {
    // ---- warps 0-7: layer 0, then every accumulator -------------------------
    // the two halves' sums, in the staging area (free until the first store)
    float* s_sum = stage;  // [2][MM]
    const int m = 32 * (warp & 3) + lane;    // tensor-memory lane = A row
    const int half = warp >> 2;              // columns [256 half, 256 half + 256)
    const long long pix = (long long)blockIdx.x * MM + m;
    const bool live = pix < npix;
    const int py = live ? (int)(pix / P.W) : 0, px = live ? (int)(pix - (long long)py * P.W) : 0;
    const float xn = live ? ((float)px - 0.5f * (float)(P.W - 1)) / (0.5f * (float)P.W) : 0.f;
    const float yn = live ? ((float)py - 0.5f * (float)(P.H - 1)) / (0.5f * (float)P.H) : 0.f;
    const float dn = live ? (P.depth[pix] - P.d_min) * P.d_scale - 1.f : 0.f;
    // layer 0's 512 {w, b} in the staging area (free until the first store):
    // one coalesced load per thread instead of 256 dependent loads each
    float4* s_wb0 = reinterpret_cast<float4*>(stage);
    for (int j = tid; j < MH; j += MEPI) s_wb0[j] = __ldg(&WB0[j]);
    named_sync_m(1, MEPI);
    for (int j0 = half * MNC; j0 < half * MNC + MNC; j0 += 8) {
      float a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = j0 + q;
        const float4 wb = s_wb0[j];
        const float v = fmaf(wb.x, xn, fmaf(wb.y, yn, fmaf(wb.z, dn, wb.w)));
        a[q] = fmaxf(v, 0.f);
      }
      *reinterpret_cast<uint4*>(Abuf + (size_t)(j0 / 8) * 2048 + m * 16) =
          make_uint4(bf2(a[0], a[1]), bf2(a[2], a[3]), bf2(a[4], a[5]), bf2(a[6], a[7]));
    }
    tc::fence_async_smem();
    tc::mbar_arrive(&s_epi[half]);
    named_sync_m(1, MEPI);  // s_wb0 is read by all before s_sum reuses the area
    float part = 0.f, sum = 0.f;
    const uint32_t tbase = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(half * MNC);
    for (int ph = 0; ph < nphase; ++ph) {
      // one thread per warp polls; its warp follows.  Half 0 of a hidden
      // layer also waits until no MMA reads inputs 0..255 any more.
      if (lane == 0) {
        mwait(&s_acc[half], (uint32_t)ph & 1u, P.status, P.wlim);
        if (half == 0 && ph < 4) mwait(&s_k0, (uint32_t)ph & 1u, P.status, P.wlim);
      }
      __syncwarp();
      tc::fence_after_sync();
      if (ph < 4) {
        const float4* bias = reinterpret_cast<const float4*>(B1 + (size_t)ph * MH + half * MNC);
        for (int c32 = 0; c32 < MNC / 32; ++c32) {
          float bb[32], v[32];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 t = __ldg(&bias[c32 * 8 + q]);
            bb[4 * q] = t.x;
            bb[4 * q + 1] = t.y;
            bb[4 * q + 2] = t.z;
            bb[4 * q + 3] = t.w;
          }
          tc::tmem_ld32(tbase + (uint32_t)(c32 * 32), v);
#pragma unroll
          for (int q = 0; q < 32; ++q) v[q] = fmaxf(v[q] + bb[q], 0.f);
          unsigned char* dst = Abuf + (size_t)((half * MNC) / 8 + c32 * 4) * 2048 + m * 16;
#pragma unroll
          for (int g = 0; g < 4; ++g)
            *reinterpret_cast<uint4*>(dst + g * 2048) =
                make_uint4(bf2(v[8 * g], v[8 * g + 1]), bf2(v[8 * g + 2], v[8 * g + 3]),
                           bf2(v[8 * g + 4], v[8 * g + 5]), bf2(v[8 * g + 6], v[8 * g + 7]));
        }
        tc::fence_async_smem();
      } else {
        const int q = mlp_pass(ph, npass), col0 = 2 * q * MNC + half * MNC;
        // columns of this half that exist (the padded rows of the output
        // layer and their biases are 0, so their outputs are exactly 0)
        const int nc32 = col0 < nout ? MNC / 32 : 0;
        const float4* bias = reinterpret_cast<const float4*>(B5 + col0);
        const bool first = ph - 4 < npass, last = ph - 4 == npass - 1;
        if (first) {  // accumulate this half's sum of clamped outputs
          for (int c32 = 0; c32 < nc32; ++c32) {
            float v[32];
            float4 bq[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) bq[g] = __ldg(&bias[c32 * 8 + g]);
            tc::tmem_ld32(tbase + (uint32_t)(c32 * 32), v);
#pragma unroll
            for (int g = 0; g < 8; ++g)
              part += (fmaxf(v[4 * g] + bq[g].x, 0.f) + fmaxf(v[4 * g + 1] + bq[g].y, 0.f)) +
                      (fmaxf(v[4 * g + 2] + bq[g].z, 0.f) + fmaxf(v[4 * g + 3] + bq[g].w, 0.f));
          }
          if (last) {  // the pixel's total: the two halves added in order
            s_sum[half * MM + m] = part;
            named_sync_m(1, MEPI);
            sum = s_sum[m] + s_sum[MM + m];
          }
        }
        if (last || !first) {  // store the pass's columns normalised
          const float inv = sum > 0.f ? 1.f / sum : 0.f;
          float* st = stage + (size_t)warp * 32 * MSROW;  // this warp's 32 pixels
          const long long wpix0 = (long long)blockIdx.x * MM + 32 * (warp & 3);
          if (last) named_sync_m(1, MEPI);  // every half has read s_sum
          for (int c32 = 0; c32 < nc32; ++c32) {
            float v[32];
            float4 bq[8];
#pragma unroll
            for (int g = 0; g < 8; ++g) bq[g] = __ldg(&bias[c32 * 8 + g]);
            tc::tmem_ld32(tbase + (uint32_t)(c32 * 32), v);
#pragma unroll
            for (int h16 = 0; h16 < 2; ++h16) {
#pragma unroll
              for (int g = 0; g < 4; ++g) {
                const float4 bb = bq[h16 * 4 + g];
                const float* vv = v + h16 * 16 + 4 * g;
                *reinterpret_cast<float2*>(st + lane * MSROW + 4 * g) =
                    make_float2(fmaxf(vv[0] + bb.x, 0.f) * inv, fmaxf(vv[1] + bb.y, 0.f) * inv);
                *reinterpret_cast<float2*>(st + lane * MSROW + 4 * g + 2) =
                    make_float2(fmaxf(vv[2] + bb.z, 0.f) * inv, fmaxf(vv[3] + bb.w, 0.f) * inv);
              }
              __syncwarp();
              // 4 pixels x 16 outputs per store: 8 lanes write one pixel's 64 bytes
              const int colc = col0 + c32 * 32 + h16 * 16 + 2 * (lane & 7);  // even
#pragma unroll
              for (int r = 0; r < 8; ++r) {
                const int pl = 4 * r + (lane >> 3);
                const long long gp = wpix0 + pl;
                if (gp < npix && colc < nout) {
                  const float2 o = *reinterpret_cast<const float2*>(st + pl * MSROW + 2 * (lane & 7));
                  const long long e = gp * (long long)nout + colc;
                  if (P.out_bf16)
                    reinterpret_cast<uint32_t*>(P.out)[e >> 1] = bf2(o.x, o.y);
                  else
                    *reinterpret_cast<float2*>(reinterpret_cast<float*>(P.out) + e) = o;
                }
              }
              __syncwarp();
            }
          }
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&s_epi[half]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 512);
}

// FP32 -> BF16 bits, round to nearest even (NaN kept quiet)
inline uint16_t host_bf16(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

}  // namespace sd

extern "C" sd_status sd_mlp_blob_bytes(int ks, size_t* bytes) {
  using namespace sd;
  if (!bytes || ks < 1 || !(ks & 1) || ks > SD_MLP_MAX_KS) return SD_ERR_ARG;
  *bytes = mlp_bytes(ks);
  return SD_OK;
}

extern "C" sd_status sd_mlp_pack(const float* const* weights, const float* const* biases, int ks,
                                 void* blob, size_t blob_bytes) {
  SD_API_RANGE("sd_mlp_pack");
  using namespace sd;
  if (!weights || !biases || !blob || ks < 1 || !(ks & 1) || ks > SD_MLP_MAX_KS) return SD_ERR_ARG;
  for (int l = 0; l < 6; ++l)
    if (!weights[l] || !biases[l]) return SD_ERR_ARG;
  if (blob_bytes < mlp_bytes(ks) || (reinterpret_cast<uintptr_t>(blob) & 255)) return SD_ERR_ARG;
  const int nout = mlp_nout(ks), nblk = mlp_nblk(ks);
  std::vector<unsigned char> host(mlp_bytes(ks), 0);
  // chunk (layer, n block, k block): element (n, k) at (k/8)*4096 + n*16 + (k%8)*2
  size_t c = 0;
  for (int l = 1; l <= 5; ++l) {
    const int rows = l < 5 ? MH : nout, nbl = l < 5 ? 2 : nblk;
    const float* Wl = weights[l];
    for (int nb = 0; nb < nbl; ++nb)
      for (int kb = 0; kb < MKPB; ++kb, ++c) {
        unsigned char* ch = host.data() + c * MCHUNK;
        for (int nl = 0; nl < MNC; ++nl)
          for (int kl = 0; kl < MKC; ++kl) {
            const int n = nb * MNC + nl, k = kb * MKC + kl;
            const uint16_t v = n < rows ? host_bf16(Wl[(size_t)n * MH + k]) : 0;
            std::memcpy(ch + (kl / 8) * 4096 + nl * 16 + (kl % 8) * 2, &v, 2);
          }
      }
  }
  float* tail = reinterpret_cast<float*>(host.data() + c * MCHUNK);
  for (int j = 0; j < MH; ++j) {
    for (int i = 0; i < 3; ++i) tail[4 * j + i] = weights[0][3 * j + i];
    tail[4 * j + 3] = biases[0][j];
  }
  for (int l = 1; l < 5; ++l) std::memcpy(tail + MH * 4 + (l - 1) * MH, biases[l], sizeof(float) * MH);
  std::memcpy(tail + MH * 8, biases[5], sizeof(float) * nout);
  SD_CUDA_TRY(cudaMemcpy(blob, host.data(), host.size(), cudaMemcpyHostToDevice));
  return SD_OK;
}

extern "C" sd_status sd_mlp_psf_map(const void* blob, int ks, const float* depth_m, int H, int W,
                                    float d_min_m, float d_max_m, void* out, int out_dtype,
                                    int32_t* status, void* stream) {
  SD_API_RANGE("sd_mlp_psf_map");
  using namespace sd;
  if (!blob || !depth_m || !out || !status || ks < 1 || !(ks & 1) || ks > SD_MLP_MAX_KS)
    return SD_ERR_ARG;
  if (H < 1 || W < 1 || !(d_max_m > d_min_m)) return SD_ERR_ARG;
  if (out_dtype != SD_F32 && out_dtype != SD_BF16) return SD_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(blob) & 255)) return SD_ERR_ARG;
  const long long npix = (long long)H * W;
  if ((npix + MM - 1) / MM > 0x7fffffffll) return SD_ERR_UNSUPPORTED;
  MlpParams P;
  P.blob = reinterpret_cast<const unsigned char*>(blob);
  P.depth = depth_m;
  P.out = out;
  P.out_bf16 = out_dtype == SD_BF16;
  P.status = reinterpret_cast<int*>(status);
  P.ks = ks;
  P.H = H;
  P.W = W;
  P.d_min = d_min_m;
  P.d_scale = 2.f / (d_max_m - d_min_m);
  P.wlim = wait_limit(MWAIT);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  SD_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
  const size_t smem = MA_BYTES + (size_t)MNB * MCHUNK + MSTAGE;
  SD_CUDA_TRY(cudaFuncSetAttribute(mlp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  mlp_kernel<<<(unsigned)((npix + MM - 1) / MM), MTHREADS, smem, s>>>(P);
  return launch_status();
}

SD_CHECK_TU(mlp)
