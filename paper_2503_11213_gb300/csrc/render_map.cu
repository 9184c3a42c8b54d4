// Per-pixel DP rendering from a PSF map (supplement, "Local DP PSF
// convolution"): every pixel (y, x) has its own kernel pair
// map[y][x][2][ks][ks], shared by all channels, and
//   out_L[n,c,y,x] = sum_{u,v} Ipad[n,c,y+u,x+v] * map[y][x][L][ks-1-u][ks-1-v]
// (likewise R), Ipad the image replicate-padded by p = (ks-1)/2.
//
// The map is read exactly once and dominates the traffic (2 ks^2 values per
// pixel against C image values), so the kernel is built around streaming it:
// one block per (8 x 32 tile, image, channel group), the tile and its halo of
// the group's channels staged in shared memory, one warp per tile row.  For
// each of its 32 pixels a warp reads the pixel's kernel pair with coalesced
// loads (the next 32*NCH values are in flight while the current ones are
// used, across pixel boundaries), multiplies each value
// with the staged image tap of every channel of the group (a per-block table
// maps a kernel index to its tap offset) and reduces over the warp; the lane
// owning the pixel keeps the sums and the row is stored coalesced at the end.
// Deterministic (fixed reduction order).

#include <cstring>

#include "common.cuh"

namespace sd {

constexpr int MT_X = 32;      // tile width (pixels) = lanes
constexpr int MT_Y = 8;       // tile height = warps per block
constexpr int MAP_NT = 32 * MT_Y;
constexpr int MAX_CP = 4;     // channels per pass
constexpr int NCH = 16;       // kernel values per lane per item

struct MapParams {
  const void* aif;
  const void* map;
  void* out;
  int N, C, H, W, ks;
  int cp;       // channels staged per pass
  int S;        // row stride of the staged tile (MT_X + ks - 1)
};

__host__ __device__ inline size_t map_smem_bytes(int ks, int cp) {
  const size_t S = MT_X + ks - 1, R = MT_Y + ks - 1;
  return (size_t)cp * S * R * 4 + (size_t)ks * ks * 4;
}

template <class TI, class TM>
__global__ void __launch_bounds__(MAP_NT) render_map_kernel(const MapParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ks = P.ks, p = (ks - 1) >> 1, ks2 = ks * ks, S = P.S, R = MT_Y + ks - 1;
  float* tile = reinterpret_cast<float*>(smem);                 // [cp][R][S]
  int* offs = reinterpret_cast<int*>(tile + (size_t)P.cp * R * S);  // [ks2]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int x0 = blockIdx.x * MT_X, y0 = blockIdx.y * MT_Y;
  const int groups = (P.C + P.cp - 1) / P.cp;
  const int n = blockIdx.z / groups, c0 = (blockIdx.z - n * groups) * P.cp;
  const int cp = min(P.cp, P.C - c0);
  const size_t plane = (size_t)P.H * P.W;

  // kernel index e = (u', v') -> offset of its tap from the pixel's staged
  // position (y - y0, x - x0): (2p - u', 2p - v') in the tile with halo p
  for (int e = tid; e < ks2; e += MAP_NT) {
    int u = e / ks, v = e - u * ks;
    offs[e] = (2 * p - u) * S + (2 * p - v);
  }
  const TI* img = reinterpret_cast<const TI*>(P.aif);
  for (int c = 0; c < cp; ++c) {
    const TI* src = img + ((size_t)n * P.C + c0 + c) * plane;
    float* dst = tile + (size_t)c * R * S;
    for (int i = tid; i < R * S; i += MAP_NT) {
      int r = i / S, q = i - r * S;
      int yy = min(max(y0 + r - p, 0), P.H - 1);
      int xx = min(max(x0 + q - p, 0), P.W - 1);
      dst[i] = to_f32<TI>(src[(size_t)yy * P.W + xx]);
    }
  }
  __syncthreads();

  const int y = y0 + warp;
  if (y >= P.H) return;
  float keep[2][MAX_CP];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int c = 0; c < MAX_CP; ++c) keep[s][c] = 0.f;
  const TM* mrow = reinterpret_cast<const TM*>(P.map) + ((size_t)y * P.W + x0) * 2 * ks2;
  const int xmax = min(MT_X, P.W - x0);
  // the row's kernels as one stream of (pixel, chunk) items of 32*NCH
  // values; the next item is loaded while the current one is used
  const int E = 2 * ks2, nchunk = (E + 32 * NCH - 1) / (32 * NCH), items = xmax * nchunk;
  const size_t RS = (size_t)R * S;
  float cur[NCH], nxt[NCH];
  auto load = [&](float* dst, int it) {
    const int px = it / nchunk, ch = it - px * nchunk;
    const TM* K = mrow + (size_t)px * E + ch * 32 * NCH;
    const int lim = E - ch * 32 * NCH;
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int e = lane + 32 * j;
      dst[j] = e < lim ? to_f32<TM>(__ldg(K + e)) : 0.f;
    }
  };
  float aL[MAX_CP], aR[MAX_CP];
#pragma unroll
  for (int c = 0; c < MAX_CP; ++c) aL[c] = aR[c] = 0.f;
  load(cur, 0);
  for (int it = 0; it < items; ++it) {
    if (it + 1 < items) load(nxt, it + 1);
    const int px = it / nchunk, ch = it - px * nchunk;
    const float* tb = tile + warp * S + px;
#pragma unroll
    for (int j = 0; j < NCH; ++j) {
      const int e = ch * 32 * NCH + lane + 32 * j;
      if (e < ks2) {
        const float* t = tb + offs[e];
#pragma unroll
        for (int c = 0; c < MAX_CP; ++c)
          if (c < cp) aL[c] = fmaf(t[c * RS], cur[j], aL[c]);
      } else if (e < E) {
        const float* t = tb + offs[e - ks2];
#pragma unroll
        for (int c = 0; c < MAX_CP; ++c)
          if (c < cp) aR[c] = fmaf(t[c * RS], cur[j], aR[c]);
      }
    }
    if (ch == nchunk - 1) {
#pragma unroll
      for (int c = 0; c < MAX_CP; ++c) {
        if (c < cp) {
          float l = aL[c], r = aR[c];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            l += __shfl_xor_sync(0xffffffffu, l, o);
            r += __shfl_xor_sync(0xffffffffu, r, o);
          }
          if (lane == px) {
            keep[0][c] = l;
            keep[1][c] = r;
          }
        }
        aL[c] = aR[c] = 0.f;
      }
    }
#pragma unroll
    for (int j = 0; j < NCH; ++j) cur[j] = nxt[j];
  }
  const int x = x0 + lane;
  if (lane < xmax) {
    TI* out = reinterpret_cast<TI*>(P.out);
#pragma unroll
    for (int c = 0; c < MAX_CP; ++c)
      if (c < cp) {
        out[(((size_t)n * 2 * P.C + c0 + c) * P.H + y) * P.W + x] = from_f32<TI>(keep[0][c]);
        out[(((size_t)n * 2 * P.C + P.C + c0 + c) * P.H + y) * P.W + x] =
            from_f32<TI>(keep[1][c]);
      }
  }
}

template <class TI, class TM>
sd_status launch_map(MapParams& P, cudaStream_t s) {
  constexpr size_t cap = 227 * 1024;
  int cp = min(MAX_CP, P.C);
  while (cp > 1 && map_smem_bytes(P.ks, cp) > cap) --cp;
  if (map_smem_bytes(P.ks, cp) > cap) return SD_ERR_UNSUPPORTED;
  P.cp = cp;
  P.S = MT_X + P.ks - 1;
  const size_t smem = map_smem_bytes(P.ks, cp);
  auto k = render_map_kernel<TI, TM>;
  SD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int groups = (P.C + cp - 1) / cp;
  if ((long long)P.N * groups > 65535) return SD_ERR_UNSUPPORTED;
  dim3 grid((P.W + MT_X - 1) / MT_X, (P.H + MT_Y - 1) / MT_Y, P.N * groups);
  k<<<grid, MAP_NT, smem, s>>>(P);
  return launch_status();
}

}  // namespace sd

extern "C" sd_status sd_dp_render_map(const void* aif, const void* psf_map, int N, int C,
                                      int H, int W, int ks, int image_dtype, int map_dtype,
                                      void* out, void* stream) {
  using namespace sd;
  if (!aif || !psf_map || !out) return SD_ERR_ARG;
  if (N < 0 || C < 1 || H < 0 || W < 0 || ks < 1 || !(ks & 1)) return SD_ERR_ARG;
  if (ks > 127) return SD_ERR_UNSUPPORTED;
  if (N == 0 || H == 0 || W == 0) return SD_OK;
  if ((long long)N * C > 65535 || (long long)H * W > (1ll << 31)) return SD_ERR_UNSUPPORTED;
  MapParams P;
  std::memset(&P, 0, sizeof P);
  P.aif = aif;
  P.map = psf_map;
  P.out = out;
  P.N = N;
  P.C = C;
  P.H = H;
  P.W = W;
  P.ks = ks;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (image_dtype == SD_F32 && map_dtype == SD_F32) return launch_map<float, float>(P, s);
  if (image_dtype == SD_F32 && map_dtype == SD_BF16) return launch_map<float, __nv_bfloat16>(P, s);
  if (image_dtype == SD_BF16 && map_dtype == SD_BF16)
    return launch_map<__nv_bfloat16, __nv_bfloat16>(P, s);
  if (image_dtype == SD_F16 && map_dtype == SD_F16) return launch_map<__half, __half>(P, s);
  if (image_dtype == SD_F32 && map_dtype == SD_F16) return launch_map<float, __half>(P, s);
  return SD_ERR_UNSUPPORTED;
}
