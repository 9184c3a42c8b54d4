// Per-pixel DP rendering from a PSF map (supplement, "Local DP PSF
// convolution"): every pixel (y, x) has its own kernel pair
// map[y][x][2][ks][ks], shared by all channels, and
//   out_L[n,c,y,x] = sum_{u,v} Ipad[n,c,y+u,x+v] * map[y][x][L][ks-1-u][ks-1-v]
// (likewise R), Ipad the image replicate-padded by p = (ks-1)/2.
//
// The map is read exactly once and dominates the traffic (2 ks^2 values per
// pixel against C image values), so the kernel is built around streaming it:
// one block per (8 x 32 tile, image, group of up to 4 channels), the tile and
// its halo staged in shared memory with the group's channels interleaved (one
// vector load per tap), one warp per tile row.  For each of its 32 pixels a
// warp reads the pixel's L and R kernels with coalesced loads (the next
// 32*NTAP taps are in flight while the current ones are used, across pixel
// boundaries); a lane takes a tap, loads the staged image values of every
// channel once and feeds both sides (a per-block table maps a tap to its
// offset); the warp reduces, and the lane owning the pixel keeps the sums,
// stored coalesced at the end.
// Deterministic (fixed reduction order).

#define SD_TU 4  // translation unit id of this file's SD_CHECK sites
#include <cstring>

#include "common.cuh"

namespace sd {

constexpr int MT_X = 32;      // tile width (pixels) = lanes
constexpr int MT_Y = 8;       // tile height = warps per block
constexpr int MAP_NT = 32 * MT_Y;
constexpr int NTAP = 8;       // taps per lane per item (L and R values each)

struct MapParams {
  const void* aif;
  const void* map;
  void* out;
  int N, C, H, W, ks;
  int S;        // row stride of the staged tile (MT_X + ks - 1), in taps
};

// CW channels interleaved per staged tap: one shared load brings all of them
template <int CW> struct Vec;
template <> struct Vec<1> { using T = float; };
template <> struct Vec<2> { using T = float2; };
template <> struct Vec<4> { using T = float4; };
__device__ __forceinline__ float comp(float v, int) { return v; }
__device__ __forceinline__ float comp(float2 v, int c) { return c == 0 ? v.x : v.y; }
__device__ __forceinline__ float comp(float4 v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

__host__ __device__ inline size_t map_smem_bytes(int ks, int cw) {
  const size_t S = MT_X + ks - 1, R = MT_Y + ks - 1;
  return (size_t)cw * S * R * 4 + (size_t)ks * ks * 4;
}

// 16-bit map values are held in registers as raw pairs and widened on use
__device__ __forceinline__ float half16(uint32_t w, int hi, __nv_bfloat16*) {
  return __uint_as_float(hi ? (w & 0xffff0000u) : (w << 16));
}
__device__ __forceinline__ float half16(uint32_t w, int hi, __half*) {
  return __half2float(__ushort_as_half((unsigned short)(hi ? (w >> 16) : (w & 0xffffu))));
}

template <class TI, class TM, int CW>
__global__ void __launch_bounds__(MAP_NT) render_map_kernel(const MapParams P) {
  using V = typename Vec<CW>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  const int ks = P.ks, p = (ks - 1) >> 1, ks2 = ks * ks, S = P.S, R = MT_Y + ks - 1;
  float* tile = reinterpret_cast<float*>(smem);                      // [R][S][CW]
  int* offs = reinterpret_cast<int*>(tile + (size_t)CW * R * S);     // [ks2]
  const V* vtile = reinterpret_cast<const V*>(tile);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int x0 = blockIdx.x * MT_X, y0 = blockIdx.y * MT_Y;
  const int groups = (P.C + CW - 1) / CW;
  const int n = blockIdx.z / groups, c0 = (blockIdx.z - n * groups) * CW;
  const int cp = min(CW, P.C - c0);
  const size_t plane = (size_t)P.H * P.W;

  // tap e = (u', v') of a kernel -> its image tap relative to the pixel's
  // staged position: (2p - u', 2p - v') in the tile with halo p
  for (int e = tid; e < ks2; e += MAP_NT) {
    int u = e / ks, v = e - u * ks;
    offs[e] = (2 * p - u) * S + (2 * p - v);
  }
  const TI* img = reinterpret_cast<const TI*>(P.aif) + ((size_t)n * P.C + c0) * plane;
  for (int i = tid; i < R * S; i += MAP_NT) {
    int r = i / S, q = i - r * S;
    int yy = min(max(y0 + r - p, 0), P.H - 1);
    int xx = min(max(x0 + q - p, 0), P.W - 1);
    const size_t src = (size_t)yy * P.W + xx;
#pragma unroll
    for (int c = 0; c < CW; ++c)
      tile[(size_t)i * CW + c] = c < cp ? to_f32<TI>(img[c * plane + src]) : 0.f;
  }
  __syncthreads();

  const int y = y0 + warp;
  if (y >= P.H) return;
  float keep[2][CW];
#pragma unroll
  for (int c = 0; c < CW; ++c) keep[0][c] = keep[1][c] = 0.f;
  const int E = 2 * ks2;
  const TM* mrow = reinterpret_cast<const TM*>(P.map) + ((size_t)y * P.W + x0) * E;
  const int xmax = min(MT_X, P.W - x0);
  // the row's kernels as a stream of (pixel, tap chunk) items of 32*NT
  // taps (L and R values of each); the next item is loaded while the current
  // one is used.  A 16-bit map moves half the bytes per load, so an item has
  // twice the taps (the same bytes in flight), kept as raw pairs.
  constexpr bool W16 = sizeof(TM) == 2;
  constexpr int NT = W16 ? 2 * NTAP : NTAP;
  constexpr int NR = W16 ? NT / 2 : NT;  // registers per plane and item
  const int nch = (ks2 + 32 * NT - 1) / (32 * NT), items = xmax * nch;
  uint32_t curL[NR], curR[NR], nxtL[NR], nxtR[NR];
  auto load = [&](uint32_t* dl, uint32_t* dr, int it) {
    const int px = it / nch, ch = it - px * nch;
    const TM* K = mrow + (size_t)px * E;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int e = ch * 32 * NT + lane + 32 * j;
      const bool in = e < ks2;
      if (W16) {
        const uint32_t l = in ? __ldg(reinterpret_cast<const unsigned short*>(K) + e) : 0u;
        const uint32_t r = in ? __ldg(reinterpret_cast<const unsigned short*>(K) + ks2 + e) : 0u;
        dl[j >> 1] = (j & 1) ? (dl[j >> 1] | (l << 16)) : l;
        dr[j >> 1] = (j & 1) ? (dr[j >> 1] | (r << 16)) : r;
      } else {
        dl[j] = __float_as_uint(in ? to_f32<TM>(__ldg(K + e)) : 0.f);
        dr[j] = __float_as_uint(in ? to_f32<TM>(__ldg(K + ks2 + e)) : 0.f);
      }
    }
  };
  auto val = [&](const uint32_t* d, int j) {
    if constexpr (W16) return half16(d[j >> 1], j & 1, (TM*)nullptr);
    else return __uint_as_float(d[j]);
  };
  float aL[CW], aR[CW];
#pragma unroll
  for (int c = 0; c < CW; ++c) aL[c] = aR[c] = 0.f;
  load(curL, curR, 0);
  for (int it = 0; it < items; ++it) {
    if (it + 1 < items) load(nxtL, nxtR, it + 1);
    const int px = it / nch, ch = it - px * nch;
    const int base = warp * S + px;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int e = ch * 32 * NT + lane + 32 * j;
      if (e < ks2 && SD_CHECK(base + offs[e], R * S)) {
        const V v = vtile[base + offs[e]];
        const float kl = val(curL, j), kr = val(curR, j);
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          aL[c] = fmaf(comp(v, c), kl, aL[c]);
          aR[c] = fmaf(comp(v, c), kr, aR[c]);
        }
      }
    }
    if (ch == nch - 1) {
#pragma unroll
      for (int c = 0; c < CW; ++c) {
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
    for (int j = 0; j < NR; ++j) {
      curL[j] = nxtL[j];
      curR[j] = nxtR[j];
    }
  }
  const int x = x0 + lane;
  if (lane < xmax) {
    TI* out = reinterpret_cast<TI*>(P.out);
#pragma unroll
    for (int c = 0; c < CW; ++c)
      if (c < cp) {
        out[(((size_t)n * 2 * P.C + c0 + c) * P.H + y) * P.W + x] = from_f32<TI>(keep[0][c]);
        out[(((size_t)n * 2 * P.C + P.C + c0 + c) * P.H + y) * P.W + x] =
            from_f32<TI>(keep[1][c]);
      }
  }
}

template <class TI, class TM, int CW>
sd_status launch_map_cw(MapParams& P, cudaStream_t s) {
  const size_t smem = map_smem_bytes(P.ks, CW);
  auto k = render_map_kernel<TI, TM, CW>;
  SD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int groups = (P.C + CW - 1) / CW;
  if ((long long)P.N * groups > 65535) return SD_ERR_UNSUPPORTED;
  dim3 grid((P.W + MT_X - 1) / MT_X, (P.H + MT_Y - 1) / MT_Y, P.N * groups);
  k<<<grid, MAP_NT, smem, s>>>(P);
  return launch_status();
}

template <class TI, class TM>
sd_status launch_map(MapParams& P, cudaStream_t s) {
  constexpr size_t cap = 227 * 1024;
  P.S = MT_X + P.ks - 1;
  // widest channel interleave that fits: 4 (RGB in one pass), 2, 1
  if (P.C > 2 && map_smem_bytes(P.ks, 4) <= cap) return launch_map_cw<TI, TM, 4>(P, s);
  if (P.C > 1 && map_smem_bytes(P.ks, 2) <= cap) return launch_map_cw<TI, TM, 2>(P, s);
  if (map_smem_bytes(P.ks, 1) <= cap) return launch_map_cw<TI, TM, 1>(P, s);
  return SD_ERR_UNSUPPORTED;
}

}  // namespace sd

extern "C" sd_status sd_dp_render_map(const void* aif, const void* psf_map, int N, int C,
                                      int H, int W, int ks, int image_dtype, int map_dtype,
                                      void* out, void* stream) {
  SD_API_RANGE("sd_dp_render_map");
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

SD_CHECK_TU(render_map)
