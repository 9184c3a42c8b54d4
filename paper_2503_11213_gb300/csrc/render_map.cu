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
#include "tc.cuh"

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

// ---------------------------------------------------------------------------
// Staged form (ks <= 21, W a multiple of the chunk's pixels, a status word):
// the same sums in the same order, with the map moved by the copy engine.
// A tile row's kernels are contiguous in the map, so each warp streams its
// row through a ring of MB_NS shared-memory stages with one-dimensional bulk
// copies (cp.async.bulk) of PC pixels each, PC * 2 ks^2 values = 16 ks^2
// bytes (PC = 4 for 16-bit maps, 2 for FP32): a multiple of 16 bytes that
// starts 16-byte aligned when W is a multiple of PC.  Lane 0 issues the
// copies, completion is counted in bytes on the stage's mbarrier, and the
// stage is refilled as soon as the warp has used it.  The kernel is
// persistent (one block per SM, the ring's size): a warp's stream runs on
// across the block's tiles, and the image tile is double-buffered, the next
// tile's values loaded into registers while the current tile is rendered.
// A warp renders a chunk's PC pixels together (independent sums) and only
// the CN channels that exist.  Per pixel, lane l takes the taps e = l + 32 j
// as the direct form with one item per pixel does, and the warp sums in the
// same butterfly, so both forms give the same bits.
// Every wait is bounded: a wait that gives up sets *err, and the warp then
// waits (bounded, not cut short) for its copies still in flight before the
// block ends.
// ---------------------------------------------------------------------------
constexpr int MB_Y = 12;                 // tile rows = warps per block
constexpr int MB_NT = 32 * MB_Y;
constexpr int MB_NS = 2;                 // ring stages per warp
constexpr int MB_NJ = 14;                // taps per lane and pixel (ks^2 <= 448)
constexpr int MB_PRE = ((MB_Y + 20) * (MT_X + 20) + MB_NT - 1) / MB_NT;  // tile values/thread
constexpr uint32_t MB_WAIT = 1u << 22;   // polls of a stage wait
constexpr uint32_t MB_DRAIN = 1u << 24;  // polls of the final drain

// esz: bytes per staged image value (4, or 2 for a 16-bit image)
__host__ __device__ inline size_t mb_smem_bytes(int ks, int cw, int esz) {
  const size_t S = MT_X + ks - 1, R = MB_Y + ks - 1;
  return (size_t)MB_Y * MB_NS * 16 * ks * ks + (size_t)2 * cw * S * R * esz;
}

// The staged image: FP32 values, or a 16-bit image's own values (widening
// them is exact, and a tap position's CW channels take half the bytes).
template <class TI, int CW> struct StageT {
  using E = float;
  using V = typename Vec<CW>::T;
};
template <int CW> struct Vec16;
template <> struct Vec16<1> { using T = unsigned short; };
template <> struct Vec16<2> { using T = ushort2; };
template <> struct Vec16<4> { using T = ushort4; };
template <int CW> struct StageT<__nv_bfloat16, CW> {
  using E = unsigned short;
  using V = typename Vec16<CW>::T;
};
template <int CW> struct StageT<__half, CW> {
  using E = unsigned short;
  using V = typename Vec16<CW>::T;
};
__device__ __forceinline__ unsigned short comp(unsigned short v, int) { return v; }
__device__ __forceinline__ unsigned short comp(ushort2 v, int c) { return c == 0 ? v.x : v.y; }
__device__ __forceinline__ unsigned short comp(ushort4 v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}
template <class TI> __device__ __forceinline__ float staged_f32(float v) { return v; }
template <class TI> __device__ __forceinline__ float staged_f32(unsigned short v);
template <> __device__ __forceinline__ float staged_f32<__nv_bfloat16>(unsigned short v) {
  return __uint_as_float((unsigned)v << 16);
}
template <> __device__ __forceinline__ float staged_f32<__half>(unsigned short v) {
  return __half2float(__ushort_as_half(v));
}
__device__ __forceinline__ float stage_value(float v) { return v; }
__device__ __forceinline__ unsigned short stage_value(__nv_bfloat16 v) {
  return __bfloat16_as_ushort(v);
}
__device__ __forceinline__ unsigned short stage_value(__half v) { return __half_as_ushort(v); }

template <class TI, class TM, int CW, int CN>
__global__ void __launch_bounds__(MB_NT, 1) render_map_bulk_kernel(const MapParams P, int ntiles,
                                                                    int* err, uint32_t wlim) {
  using SE = typename StageT<TI, CW>::E;  // a staged image value
  using V = typename StageT<TI, CW>::V;
  constexpr int PC = 8 / (int)sizeof(TM);  // pixels per chunk
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_bar[MB_Y][MB_NS];
  const int ks = P.ks, p = (ks - 1) >> 1, ks2 = ks * ks, S = P.S, R = MB_Y + ks - 1;
  const int E = 2 * ks2, RS = R * S;
  const uint32_t CHB = 16u * (uint32_t)ks2;  // bytes per chunk
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned char* ring = smem + (size_t)warp * MB_NS * CHB;
  SE* tiles = reinterpret_cast<SE*>(smem + (size_t)MB_Y * MB_NS * CHB);  // [2][R][S][CW]
  const int ntx = (P.W + MT_X - 1) / MT_X, nty = (P.H + MB_Y - 1) / MB_Y;
  const int groups = (P.C + CW - 1) / CW;
  const size_t plane = (size_t)P.H * P.W;

  // staged-tile offset of the lane's taps e = lane + 32 j: kernel element
  // (u', v') meets the image at (2p - u', 2p - v') from the pixel's position
  int offj[MB_NJ];
#pragma unroll
  for (int j = 0; j < MB_NJ; ++j) {
    const int e = lane + 32 * j, u = e / ks, v = e - u * ks;
    offj[j] = (2 * p - u) * S + (2 * p - v);
  }
  if (tid == 0) {
    for (int w = 0; w < MB_Y; ++w)
      for (int b = 0; b < MB_NS; ++b) tc::mbar_init(&s_bar[w][b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  // the image tile of tile t (replicate padding by clamping), CW channels
  // interleaved: thread values first (registers), then the shared buffer
  SE pre[MB_PRE][CW];
  auto tile_load = [&](int t) {
    const int bx = t % ntx, r = t / ntx, by = r % nty, z = r / nty;
    const int n = z / groups, c0 = (z - n * groups) * CW, cp = min(CW, P.C - c0);
    const TI* img = reinterpret_cast<const TI*>(P.aif) + ((size_t)n * P.C + c0) * plane;
#pragma unroll
    for (int k = 0; k < MB_PRE; ++k) {
      const int i = tid + k * MB_NT;
      const int rr = i / S, q = i - rr * S;
      const int yy = min(max(by * MB_Y + rr - p, 0), P.H - 1);
      const int xx = min(max(bx * MT_X + q - p, 0), P.W - 1);
      const size_t src = (size_t)yy * P.W + xx;
#pragma unroll
      for (int c = 0; c < CW; ++c)
        pre[k][c] = (i < RS && c < cp) ? stage_value(img[c * plane + src]) : SE(0);
    }
  };
  auto tile_store = [&](SE* dst) {
#pragma unroll
    for (int k = 0; k < MB_PRE; ++k) {
      const int i = tid + k * MB_NT;
      if (i < RS) {
#pragma unroll
        for (int c = 0; c < CW; ++c) dst[(size_t)i * CW + c] = pre[k][c];
      }
    }
  };
  if (blockIdx.x < ntiles) {
    tile_load(blockIdx.x);
    tile_store(tiles);
  }
  __syncthreads();

  // the warp's chunk stream: for each tile t of the block (t = blockIdx.x,
  // + gridDim.x, ...) the chunks of the warp's row; lane 0 issues them
  int pt = blockIdx.x, pc = 0, issued = 0;
  auto issue_next = [&]() {
    while (pt < ntiles) {
      const int bx = pt % ntx, by = (pt / ntx) % nty;
      const int y = by * MB_Y + warp, x0 = bx * MT_X;
      const int nck = y < P.H ? min(MT_X, P.W - x0) / PC : 0;
      if (pc < nck) {
        const int b = issued % MB_NS;
        const TM* src = reinterpret_cast<const TM*>(P.map) +
                        ((size_t)y * P.W + x0 + (size_t)pc * PC) * E;
        tc::mbar_arrive_expect_tx(&s_bar[warp][b], CHB);
        tc::bulk_g2s(ring + (size_t)b * CHB, src, CHB, &s_bar[warp][b]);
        ++issued;
        ++pc;
        return;
      }
      pt += gridDim.x;
      pc = 0;
    }
  };
  if (lane == 0)
    for (int i = 0; i < MB_NS; ++i) issue_next();
  int done = 0;    // chunks received
  bool ok = true;  // no wait of this warp gave up

  for (int t = blockIdx.x, cur = 0; t < ntiles; t += gridDim.x, cur ^= 1) {
    const int bx = t % ntx, r = t / ntx, by = r % nty, z = r / nty;
    const int n = z / groups, c0 = (z - n * groups) * CW, cp = min(CW, P.C - c0);
    const int x0 = bx * MT_X, y = by * MB_Y + warp;
    const bool next = t + (int)gridDim.x < ntiles;
    if (next) tile_load(t + gridDim.x);  // in flight during this tile
    const V* vtile = reinterpret_cast<const V*>(tiles + (size_t)cur * RS * CW);
    if (y < P.H) {  // warp-uniform
      const int xmax = min(MT_X, P.W - x0), nck = xmax / PC;
      float keep[2][CN];
#pragma unroll
      for (int c = 0; c < CN; ++c) keep[0][c] = keep[1][c] = 0.f;
      for (int ci = 0; ci < nck && ok; ++ci) {
        const int b = done % MB_NS;
        const bool got = __all_sync(0xffffffffu, tc::mbar_wait(&s_bar[warp][b],
                                                               (uint32_t)(done / MB_NS) & 1u,
                                                               wlim, err));
        if (!got) {
          if (lane == 0) atomicExch(err, 1);
          ok = false;
          break;
        }
        ++done;
        const TM* K0 = reinterpret_cast<const TM*>(ring + (size_t)b * CHB);
        const int base = warp * S + ci * PC;
        float aL[PC][CN], aR[PC][CN];
#pragma unroll
        for (int q = 0; q < PC; ++q)
#pragma unroll
          for (int c = 0; c < CN; ++c) aL[q][c] = aR[q][c] = 0.f;
#pragma unroll
        for (int j = 0; j < MB_NJ; ++j) {
          const int e = lane + 32 * j;
          if (e < ks2) {
#pragma unroll
            for (int q = 0; q < PC; ++q) {
              if (!SD_CHECK(base + q + offj[j], RS)) continue;
              const V v = vtile[base + q + offj[j]];
              const float kl = to_f32<TM>(K0[q * E + e]), kr = to_f32<TM>(K0[q * E + ks2 + e]);
#pragma unroll
              for (int c = 0; c < CN; ++c) {
                const float iv = staged_f32<TI>(comp(v, c));
                aL[q][c] = fmaf(iv, kl, aL[q][c]);
                aR[q][c] = fmaf(iv, kr, aR[q][c]);
              }
            }
          }
        }
        // the stage's reads are done: refill it (async-proxy writes after
        // generic-proxy reads), then the warp sums
        __syncwarp();
        if (lane == 0) {
          tc::fence_async_smem();
          issue_next();
        }
        // the warp sums of the chunk's NV values (pixel, side, channel
        // padded to CP) by recursive halving: at offset o a lane keeps half
        // of its values and adds the partner's copies of them, the pairs of
        // the butterfly that every lane would run on every value (the same
        // sums); value k ends in lanes k << (5 - log2 NV) ...
        constexpr int CP = CN == 3 ? 4 : CN, NV = PC * 2 * CP;
        constexpr int LV = NV >= 32 ? 5 : NV >= 16 ? 4 : NV >= 8 ? 3 : NV >= 4 ? 2 : 1;
        float w[NV];
#pragma unroll
        for (int q = 0; q < PC; ++q)
#pragma unroll
          for (int c = 0; c < CP; ++c) {
            w[(q * 2) * CP + c] = c < CN ? aL[q][c < CN ? c : 0] : 0.f;
            w[(q * 2 + 1) * CP + c] = c < CN ? aR[q][c < CN ? c : 0] : 0.f;
          }
#pragma unroll
        for (int lv = 0; lv < 5; ++lv) {
          const int o = 16 >> lv, n = NV >> lv;
          if (lv < LV) {
            const bool hi = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < n / 2; ++i) {
              const float snd = hi ? w[i] : w[i + n / 2];
              const float kp = hi ? w[i + n / 2] : w[i];
              w[i] = kp + __shfl_xor_sync(0xffffffffu, snd, o);
            }
          } else {
            w[0] += __shfl_xor_sync(0xffffffffu, w[0], o);
          }
        }
        // ... from where the lane of pixel ci * PC + q takes its 2 CN sums
        const int qq = lane - ci * PC;
        const bool mine = qq >= 0 && qq < PC;
#pragma unroll
        for (int sd2 = 0; sd2 < 2; ++sd2)
#pragma unroll
          for (int c = 0; c < CN; ++c) {
            const int k = ((mine ? qq : 0) * 2 + sd2) * CP + c;
            const float v = __shfl_sync(0xffffffffu, w[0], k << (5 - LV));
            if (mine) keep[sd2][c] = v;
          }
      }
      if (ok && lane < xmax) {
        TI* out = reinterpret_cast<TI*>(P.out);
        const int x = x0 + lane;
#pragma unroll
        for (int c = 0; c < CN; ++c)
          if (c < cp) {
            out[(((size_t)n * 2 * P.C + c0 + c) * P.H + y) * P.W + x] = from_f32<TI>(keep[0][c]);
            out[(((size_t)n * 2 * P.C + P.C + c0 + c) * P.H + y) * P.W + x] =
                from_f32<TI>(keep[1][c]);
          }
      }
    }
    if (next) tile_store(tiles + (size_t)(cur ^ 1) * RS * CW);
    __syncthreads();  // the next tile is staged; this tile's reads are done
  }
  // no copy may still be landing when the block ends: after an error the
  // warp waits (bounded) for the chunks it issued and did not receive
  if (lane == 0)
    for (int sq = done; sq < issued; ++sq)
      if (!tc::mbar_wait(&s_bar[warp][sq % MB_NS], (uint32_t)(sq / MB_NS) & 1u, MB_DRAIN))
        atomicExch(err, 1);
}

template <class TI, class TM, int CW, int CN>
sd_status launch_map_bulk(MapParams& P, int* err, cudaStream_t s) {
  const size_t smem = mb_smem_bytes(P.ks, CW, (int)sizeof(typename StageT<TI, CW>::E));
  auto k = render_map_bulk_kernel<TI, TM, CW, CN>;
  SD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0, occ = 0;
  SD_CUDA_TRY(cudaGetDevice(&dev));
  SD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  SD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, MB_NT, smem));
  const long long ntiles = (long long)((P.W + MT_X - 1) / MT_X) * ((P.H + MB_Y - 1) / MB_Y) *
                           P.N * ((P.C + CW - 1) / CW);
  if (ntiles > 0x7fffffffll) return SD_ERR_UNSUPPORTED;
  const long long grid = std::min(ntiles, (long long)nsm * std::max(occ, 1));
  k<<<(unsigned)grid, MB_NT, smem, s>>>(P, (int)ntiles, err, wait_limit(MB_WAIT));
  return launch_status();
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
sd_status launch_map(MapParams& P, int* err, cudaStream_t s) {
  constexpr size_t cap = 227 * 1024;
  P.S = MT_X + P.ks - 1;
  // the staged form when its chunks are 16-byte aligned and the ring fits
  constexpr int PC = 8 / (int)sizeof(TM);
  if (err && P.ks * P.ks <= 32 * MB_NJ && P.W % PC == 0 &&
      (reinterpret_cast<uintptr_t>(P.map) & 15) == 0) {
    const int esz = sizeof(TI) == 2 ? 2 : 4;
    if (P.C == 3 && mb_smem_bytes(P.ks, 4, esz) <= cap)
      return launch_map_bulk<TI, TM, 4, 3>(P, err, s);
    if (P.C > 3 && mb_smem_bytes(P.ks, 4, esz) <= cap)
      return launch_map_bulk<TI, TM, 4, 4>(P, err, s);
    if (P.C == 2 && mb_smem_bytes(P.ks, 2, esz) <= cap)
      return launch_map_bulk<TI, TM, 2, 2>(P, err, s);
    if (mb_smem_bytes(P.ks, 1, esz) <= cap) return launch_map_bulk<TI, TM, 1, 1>(P, err, s);
  }
  // widest channel interleave that fits: 4 (RGB in one pass), 2, 1
  if (P.C > 2 && map_smem_bytes(P.ks, 4) <= cap) return launch_map_cw<TI, TM, 4>(P, s);
  if (P.C > 1 && map_smem_bytes(P.ks, 2) <= cap) return launch_map_cw<TI, TM, 2>(P, s);
  if (map_smem_bytes(P.ks, 1) <= cap) return launch_map_cw<TI, TM, 1>(P, s);
  return SD_ERR_UNSUPPORTED;
}

}  // namespace sd

extern "C" sd_status sd_dp_render_map(const void* aif, const void* psf_map, int N, int C,
                                      int H, int W, int ks, int image_dtype, int map_dtype,
                                      void* out, int32_t* status, void* stream) {
  SD_API_RANGE("sd_dp_render_map");
  using namespace sd;
  if (!aif || !psf_map || !out) return SD_ERR_ARG;
  if (N < 0 || C < 1 || H < 0 || W < 0 || ks < 1 || !(ks & 1)) return SD_ERR_ARG;
  if (ks > 127) return SD_ERR_UNSUPPORTED;
  const bool f32i = image_dtype == SD_F32;
  if (!((f32i && (map_dtype == SD_F32 || map_dtype == SD_BF16 || map_dtype == SD_F16)) ||
        (image_dtype == SD_BF16 && map_dtype == SD_BF16) ||
        (image_dtype == SD_F16 && map_dtype == SD_F16)))
    return SD_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* err = reinterpret_cast<int*>(status);
  if (err) SD_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
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
  if (f32i && map_dtype == SD_F32) return launch_map<float, float>(P, err, s);
  if (f32i && map_dtype == SD_BF16) return launch_map<float, __nv_bfloat16>(P, err, s);
  if (image_dtype == SD_BF16) return launch_map<__nv_bfloat16, __nv_bfloat16>(P, err, s);
  if (image_dtype == SD_F16) return launch_map<__half, __half>(P, err, s);
  return launch_map<float, __half>(P, err, s);
}

SD_CHECK_TU(render_map)
