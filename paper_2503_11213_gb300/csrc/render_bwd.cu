// Adjoint of the per-pixel DP render (supplement, "Local DP PSF convolution").
//
// Forward (bank mode): out_s(y,x) = sum_{u,v} Ipad(y+u, x+v) Kf_s(y,x)[u][v],
// side s in {L, R}, Kf = the pixel's kernel flipped in both axes, and the
// kernel a two-slice blend K = (1-t) B[key] + t B[key+1].  With G_s = dLoss/
// dout_s the adjoints are
//   dIpad(y+u, x+v) += sum_s G_s(y,x) Kf_s(y,x)[u][v]      (then the replicate
//                      padding folds every padded position onto its clamped
//                      source pixel),
//   dB[key][s][ks-1-u][ks-1-v] += sum_{pixels using key} w(y,x) G_s(y,x)
//                      Ipad(y+u, x+v)   with w = 1-t or t.
// Three kernels:
//   slice_bitmap_kernel     per (image, tile): which bank slices the tile uses
//                           (a bitmap in the caller's workspace);
//   render_bwd_img_kernel   per (tile, channel): the forward's work list of
//                           (segment, slice) items; each lane scatters its
//                           segment's weighted gradients through a register
//                           window of 8 taps into a shared padded tile, which
//                           is then folded into grad_aif with global atomics
//                           (FP32 addition order varies: not bitwise
//                           reproducible);
//   render_bwd_bank_kernel  per (slice, wavelength): visits, in a fixed order,
//                           the tiles whose bitmap holds the slice; threads own
//                           8-tap strips of the kernel and accumulate over the
//                           tile's segments in a fixed order: deterministic.

#include <algorithm>
#include <mutex>

#include "render_common.cuh"
#include "tc.cuh"

namespace sd {

constexpr int TXB = 64;            // tile width of the bitmap / bank-gradient pass
constexpr int NT_BM = 256;         // threads of the bitmap kernel (= TXB*RT_Y/SEG)

inline size_t bitmap_words(int nkeys) { return ((size_t)nkeys + 31) / 32; }

inline void bwd_tiles(int H, int W, int* tx, int* ty) {
  *tx = (W + TXB - 1) / TXB;
  *ty = (H + RT_Y - 1) / RT_Y;
}

// ---------------------------------------------------------------------------
// 1. slice bitmap per (image, tile)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT_BM) slice_bitmap_kernel(const RenderParams P,
                                                             unsigned* __restrict__ bm,
                                                             int words) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned* sb = reinterpret_cast<unsigned*>(smem);
  const int tid = threadIdx.x;
  for (int i = tid; i < words; i += NT_BM) sb[i] = 0u;
  __syncthreads();
  const int n = blockIdx.z, tx0 = blockIdx.x * TXB, ty0 = blockIdx.y * RT_Y;
  const int col = tid % TXB, rb = tid / TXB;
  const bool two = P.Z > 1;
  for (int j = 0; j < SEG; ++j) {
    int yy = ty0 + rb * SEG + j, xx = tx0 + col;
    if (yy >= P.H || xx >= P.W) continue;
    int key;
    float t;
    select_slice(P, yy, xx, P.depth[((size_t)n * P.H + yy) * P.W + xx], &key, &t);
    if (!two || t < 1.f) atomicOr(&sb[key >> 5], 1u << (key & 31));
    if (two && t > 0.f) atomicOr(&sb[(key + 1) >> 5], 1u << ((key + 1) & 31));
  }
  __syncthreads();
  size_t tile = ((size_t)n * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  for (int i = tid; i < words; i += NT_BM) bm[tile * words + i] = sb[i];
}

// ---------------------------------------------------------------------------
// 2. image gradient.  Each lane owns a vertical segment of SB pixels; every
// shared-memory atomic carries 2*SB FMAs.
// ---------------------------------------------------------------------------
template <int TX, int VB, int SB>
struct BwdImgSmem {
  static constexpr int NT = TX * RT_Y / SB, NW = NT / 32, NPX = TX * RT_Y, MW = NT / 32;
  __host__ __device__ static int ku(int ks) { return (ks + SB - 1) / SB * SB; }
  __host__ __device__ static size_t kbuf_words(int ks) { return (size_t)2 * (2 * ku(ks) * VB); }
  __host__ __device__ static size_t pad_words(int ks) {
    return (size_t)(TX + ks - 1) * (RT_Y + ks - 1 + SB);
  }
  static size_t bytes(int ks) {
    size_t w = pad_words(ks) + NW * kbuf_words(ks) + 3 * (size_t)NPX  // dIpad, K, gL/gR, t
               + (size_t)RK * MW + (RK + 1) + MAX_CHUNKS + NPX / 2;
    return 4 * w;
  }
};

template <int TX, int VB, int KSMAX, int SB, class TB>
__global__ void __launch_bounds__(TX * RT_Y / SB, 1)
    render_bwd_img_kernel(const RenderParams P, const float* __restrict__ gout,
                          float* __restrict__ gaif) {
  using SM = BwdImgSmem<TX, VB, SB>;
  constexpr int NT = SM::NT, NW = SM::NW, NPX = SM::NPX, MW = SM::MW;
  constexpr int NR = (2 * ((KSMAX + SB - 1) / SB * SB) * VB + 31) / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const int ks = P.ks, p = (ks - 1) >> 1, ks2 = ks * ks;
  const int S = P.halo_w;
  float* dpad = reinterpret_cast<float*>(smem);
  float* kbuf = dpad + SM::pad_words(ks);
  float* gL = kbuf + NW * SM::kbuf_words(ks);
  float* gR = gL + NPX;
  float* pt = gR + NPX;
  unsigned* mask = reinterpret_cast<unsigned*>(pt + NPX);
  int* kpre = reinterpret_cast<int*>(mask + RK * MW);
  int* chunks = kpre + RK + 1;
  unsigned short* prel = reinterpret_cast<unsigned short*>(chunks + MAX_CHUNKS);
  __shared__ int s_kmin, s_kmax, s_nchunks, s_next;

  const int tx0 = blockIdx.x * TX, ty0 = blockIdx.y * RT_Y;
  const int n = blockIdx.z / P.C, c = blockIdx.z - n * P.C;
  const int lam = (P.NL == P.C) ? c : 0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int H = P.H, W = P.W;
  const bool two = (P.Z > 1);

  const int seg_col = tid % TX, seg_rb = tid / TX;
  int kmin_t = 0x7fffffff, kmax_t = -1;
  int key_j[SB];
  float t_j[SB];
  const float* goL = gout + (((size_t)n * 2 * P.C + c) * H) * W;
  const float* goR = gout + (((size_t)n * 2 * P.C + P.C + c) * H) * W;
#pragma unroll
  for (int j = 0; j < SB; ++j) {
    int yy = ty0 + seg_rb * SB + j, xx = tx0 + seg_col;
    int pix = (seg_rb * SB + j) * TX + seg_col;
    key_j[j] = -1;
    t_j[j] = 0.f;
    float a = 0.f, b = 0.f;
    if (yy < H && xx < W) {
      float d = P.depth[((size_t)n * H + yy) * W + xx];
      select_slice(P, yy, xx, d, &key_j[j], &t_j[j]);
      kmin_t = min(kmin_t, key_j[j]);
      kmax_t = max(kmax_t, key_j[j] + (two ? 1 : 0));
      a = goL[(size_t)yy * W + xx];
      b = goR[(size_t)yy * W + xx];
    }
    pt[pix] = t_j[j];
    gL[pix] = a;
    gR[pix] = b;
  }
  if (tid == 0) {
    s_kmin = 0x7fffffff;
    s_kmax = -1;
  }
  for (int i = tid; i < (int)SM::pad_words(ks); i += NT) dpad[i] = 0.f;
  __syncthreads();
  atomicMin(&s_kmin, kmin_t);
  atomicMax(&s_kmax, kmax_t);
  __syncthreads();
  const int kmin = s_kmin, kmax = s_kmax;
#pragma unroll
  for (int j = 0; j < SB; ++j)
    prel[(seg_rb * SB + j) * TX + seg_col] =
        (unsigned short)(key_j[j] >= 0 ? key_j[j] - kmin : 0xffff);

  float* kb = kbuf + warp * SM::kbuf_words(ks);
  const int nblk = (ks + VB - 1) / VB;
  const int KU = SM::ku(ks);
  const int kb_elems = 2 * KU * VB;

  for (int wbase = kmin; wbase <= kmax; wbase += RK) {
    for (int i = tid; i < RK * MW; i += NT) mask[i] = 0u;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SB; ++j) {
      int k0 = key_j[j];
      if (k0 < 0) continue;
      float t = t_j[j];
      if ((!two || t < 1.f) && k0 >= wbase && k0 < wbase + RK)
        atomicOr(&mask[(k0 - wbase) * MW + warp], 1u << lane);
      if (two && t > 0.f && k0 + 1 >= wbase && k0 + 1 < wbase + RK)
        atomicOr(&mask[(k0 + 1 - wbase) * MW + warp], 1u << lane);
    }
    __syncthreads();
    if (warp == 0) {
      int carry = 0;
      for (int k0 = 0; k0 < RK; k0 += 32) {
        int k = k0 + lane;
        int cnt = 0;
        for (int w = 0; w < MW; ++w) cnt += __popc(mask[k * MW + w]);
        int nch = (cnt + 31) >> 5;
        int v = nch;
        for (int o = 1; o < 32; o <<= 1) {
          int u = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += u;
        }
        kpre[k] = carry + v - nch;
        carry += __shfl_sync(0xffffffffu, v, 31);
      }
      if (lane == 0) {
        kpre[RK] = carry;
        s_nchunks = carry;
      }
    }
    __syncthreads();
    const int nchunks = s_nchunks;
    for (int k = tid; k < RK; k += NT)
      for (int q = kpre[k]; q < kpre[k + 1]; ++q) chunks[q] = (k << 8) | (q - kpre[k]);
    if (tid == 0) s_next = NW;
    __syncthreads();

    for (int ch = warp; ch < nchunks;) {
      const int rel = chunks[ch] >> 8, sub = chunks[ch] & 0xff;
      const int key = wbase + rel;
      int want = sub * 32 + lane, seg = -1;
      for (int w = 0; w < MW; ++w) {
        unsigned m = mask[rel * MW + w];
        int pc = __popc(m);
        if (seg < 0 && want >= 0 && want < pc) {
          for (int q = 0; q < want; ++q) m &= m - 1;
          seg = w * 32 + __ffs(m) - 1;
        }
        want -= pc;
      }
      const bool act = seg >= 0;
      const int sg = act ? seg : 0;
      const int col = sg % TX, rb = sg / TX;
      // weighted gradients of the segment's pixels for this slice
      float GL[SB], GR[SB];
#pragma unroll
      for (int j = 0; j < SB; ++j) {
        int pix = (rb * SB + j) * TX + col;
        unsigned short r16 = prel[pix];
        float w = 0.f;
        if (act && r16 != 0xffff) {
          int k0 = kmin + (int)r16;
          float t = pt[pix];
          w = (k0 == key) ? (two ? 1.f - t : 1.f) : ((two && k0 + 1 == key) ? t : 0.f);
        }
        GL[j] = w * gL[pix];
        GR[j] = w * gR[pix];
      }
      const int f = key / P.Z, z = key - f * P.Z;
      // quadrant bank: field cell and flips (x: mirror columns and exchange
      // L and R; y: mirror rows); radial bank: flips = 0
      const int flips = f / P.FC, cell = f - flips * P.FC;
      const TB* K0 = reinterpret_cast<const TB*>(P.bank) +
                     (((size_t)cell * P.Z + z) * P.NL + lam) * 2 * ks2;
      const TB* KL = (flips & 1) ? K0 + ks2 : K0;
      const TB* KR = (flips & 1) ? K0 : K0 + ks2;
      const bool mx = flips & 1, my = flips & 2;
      float pre[NR];
      auto fetch = [&](int b) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          int e = lane + 32 * r;
          float v = 0.f;
          if (e < kb_elems) {
            int side = e & 1, uv = e >> 1, u = uv / VB, vv = uv - u * VB;
            int v_ = b * VB + vv;
            if (v_ < ks && u < ks)
              v = to_f32<TB>(__ldg((side ? KR : KL) + (my ? u : ks - 1 - u) * ks +
                                   (mx ? v_ : ks - 1 - v_)));
          }
          pre[r] = v;
        }
      };
      auto commit = [&](float* dst) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          int e = lane + 32 * r;
          if (e < kb_elems) dst[e] = pre[r];
        }
      };
      // rows [ulo, uhi] of the fetched block holding a non-zero tap
      auto extent = [&](int& ulo, int& uhi) {
        unsigned lo_l = 0xffffffffu, hi_l = 0u;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          int e = lane + 32 * r;
          if (e < kb_elems && pre[r] != 0.f) {
            unsigned u = (unsigned)((e >> 1) / VB);
            lo_l = min(lo_l, u);
            hi_l = max(hi_l, u + 1u);
          }
        }
        ulo = (int)__reduce_min_sync(0xffffffffu, lo_l);
        uhi = (int)__reduce_max_sync(0xffffffffu, hi_l) - 1;
      };
      int ulo_n, uhi_n;
      fetch(0);
      extent(ulo_n, uhi_n);
      commit(kb);
      __syncwarp();
      float* base = dpad + (rb * SB) * S + col;
      for (int b = 0; b < nblk; ++b) {
        const float* kcur = kb + (b & 1) * kb_elems;
        const int ulo = ulo_n, uhi = uhi_n;
        if (b + 1 < nblk) fetch(b + 1);
        // taps outside rows [ulo, uhi] are zero: padded rows r in
        // [r_begin, uhi + SB) are the only ones that can receive anything
        const int r_begin = (ulo / SB) * SB;
        const int vmax = uhi < 0 ? 0 : min(VB, ks - b * VB);
        for (int vv = 0; vv < vmax; ++vv) {
          float* colp = base + b * VB + vv;
          const float2* kp = reinterpret_cast<const float2*>(kcur) + vv;
          // ring of the taps u = r-SB+1 .. r of column v (zero outside [0, ks))
          float kl[SB], kr[SB];
#pragma unroll
          for (int j = 0; j < SB; ++j) kl[j] = kr[j] = 0.f;
          // contribution to padded row rb*SB + r: sum_j G_j Kf[r-j].  Rows
          // r < KU: every tap row exists and every padded row is in the tile
          // (KU <= ks + SB - 1); rows KU .. KU+SB-1 only drain the ring into
          // the rows below ks + SB - 1.
          const float2* kq = kp + r_begin * VB;
          float* dq = colp + r_begin * S;
          for (int r0 = r_begin; r0 < uhi + SB; r0 += SB) {
            const bool tail = r0 >= KU;
#pragma unroll
            for (int q = 0; q < SB; ++q) {
              const float2 w2 = tail ? make_float2(0.f, 0.f) : kq[q * VB];
              kl[q] = w2.x;
              kr[q] = w2.y;
              float a4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
              for (int jj = 0; jj < SB; ++jj) {
                a4[jj & 3] = fmaf(GL[jj], kl[(q - jj + SB) % SB], a4[jj & 3]);
                a4[jj & 3] = fmaf(GR[jj], kr[(q - jj + SB) % SB], a4[jj & 3]);
              }
              // zero taps are common (the L and R halves of a blur disc),
              // and skipping their atomics is what sets this loop's speed
              const float acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
              if ((!tail || r0 + q < ks + SB - 1) && acc != 0.f) atomicAdd(dq + q * S, acc);
            }
            kq += SB * VB;
            dq += SB * S;
          }
        }
        if (b + 1 < nblk) {
          extent(ulo_n, uhi_n);
          commit(kb + ((b + 1) & 1) * kb_elems);
        }
        __syncwarp();
      }
      int nxt = 0;
      if (lane == 0) nxt = atomicAdd(&s_next, 1);
      ch = __shfl_sync(0xffffffffu, nxt, 0);
    }
    __syncthreads();
  }
  // fold the padded tile onto the image (replicate padding adjoint)
  float* ga = gaif + ((size_t)n * P.C + c) * H * W;
  for (int i = tid; i < P.halo_h * S; i += NT) {
    float v = dpad[i];
    if (v == 0.f) continue;
    int r = i / S, cc = i - r * S;
    int yy = min(max(ty0 + r - p, 0), H - 1);
    int xx = min(max(tx0 + cc - p, 0), W - 1);
    atomicAdd(&ga[(size_t)yy * W + xx], v);
  }
}

// ---------------------------------------------------------------------------
// 3. bank gradient, one block per (slice key, wavelength)
// ---------------------------------------------------------------------------
// The tiles t0 .. t0 + NT - 1 (of ntiles) of this block's part whose bitmap
// holds the slice, as offsets from t0 in ascending order: one tile per
// thread, compacted with warp ballots, so that the bitmap loads of NT tiles
// are in flight together (a scan of one tile after the other waits for each
// load in turn).  Every thread of the block calls it; returns the count.
template <int NT>
__device__ int slice_tiles(const unsigned* __restrict__ bm, int words, int kw, unsigned kbit,
                           size_t t0, size_t ntiles, int parts, int part, int* s_list,
                           int* s_wc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t t = t0 + tid;
  const bool use =
      t < ntiles && (int)(t % (size_t)parts) == part && (bm[t * words + kw] & kbit) != 0u;
  const unsigned bal = __ballot_sync(0xffffffffu, use);
  if (lane == 0) s_wc[warp] = __popc(bal);
  __syncthreads();
  int pos = __popc(bal & ((1u << lane) - 1u)), tot = 0;
  for (int w = 0; w < NT / 32; ++w) {
    const int c = s_wc[w];
    pos += w < warp ? c : 0;
    tot += c;
  }
  if (use) s_list[pos] = tid;
  __syncthreads();
  return tot;
}

template <int NT, int SPT, class TI>
__global__ void __launch_bounds__(NT, NT <= 256 ? 3 : 1) render_bwd_bank_kernel(const RenderParams P,
                                                             const float* __restrict__ gout,
                                                             const unsigned* __restrict__ bm,
                                                             int words, int ntx, int nty,
                                                             float* __restrict__ gbank,
                                                             int parts) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ks = P.ks, p = (ks - 1) >> 1, ks2 = ks * ks;
  const int KU = (ks + SEG - 1) / SEG * SEG;
  const int S = TXB + ks - 1;
  const int HH = RT_Y + ks - 1 + SEG;
  constexpr int NPX = TXB * RT_Y, NSEG = NPX / SEG;
  // one thread per segment builds the segment list below
  static_assert(NT >= NSEG, "the bank-gradient block needs a thread per segment");
  float* halo = reinterpret_cast<float*>(smem);          // HH x S
  float2* G = reinterpret_cast<float2*>(halo + (size_t)HH * S);  // NPX (L, R)
  int* segs = reinterpret_cast<int*>(G + NPX);            // NSEG
  __shared__ int s_nseg, s_wcnt[NSEG / 32];

  // block (key, lam, part) visits the tiles with index = part (mod parts)
  const int key = blockIdx.x, lam = blockIdx.y, part = blockIdx.z;
  const int tid = threadIdx.x;
  const bool two = P.Z > 1;
  const int nstrip = ks * (KU / SEG);
  float acc[SPT][2 * SEG];
#pragma unroll
  for (int s = 0; s < SPT; ++s)
#pragma unroll
    for (int i = 0; i < 2 * SEG; ++i) acc[s][i] = 0.f;

  const int kw = key >> 5;
  const unsigned kbit = 1u << (key & 31);
  const int c_lo = (P.NL == P.C) ? lam : 0, c_hi = (P.NL == P.C) ? lam + 1 : P.C;
  // the tiles of this part that use the slice, in ascending order
  __shared__ int s_list[NT], s_twc[NT / 32];
  const size_t ntiles = (size_t)P.N * nty * ntx;
  for (size_t t0 = 0; t0 < ntiles; t0 += NT)
    for (int li = 0, nlist = slice_tiles<NT>(bm, words, kw, kbit, t0, ntiles, parts, part,
                                             s_list, s_twc);
         li < nlist; ++li) {
        const size_t tile = t0 + s_list[li];
        const int n = (int)(tile / ((size_t)nty * ntx));
        const int rem = (int)(tile - (size_t)n * nty * ntx);
        const int ty = rem / ntx, tx = rem - ty * ntx;
        const int tx0 = tx * TXB, ty0 = ty * RT_Y;
        for (int c = c_lo; c < c_hi; ++c) {
          __syncthreads();
          const TI* img = reinterpret_cast<const TI*>(P.aif) + ((size_t)n * P.C + c) * P.H * P.W;
          // one warp per halo row (no division by the runtime row length)
          for (int r = tid >> 5; r < HH; r += NT / 32) {
            const TI* src = img + (size_t)min(max(ty0 + r - p, 0), P.H - 1) * P.W;
#pragma unroll 4
            for (int cc = tid & 31; cc < S; cc += 32)
              halo[r * S + cc] = to_f32<TI>(src[min(max(tx0 + cc - p, 0), P.W - 1)]);
          }
          const float* goL = gout + (((size_t)n * 2 * P.C + c) * P.H) * P.W;
          const float* goR = gout + (((size_t)n * 2 * P.C + P.C + c) * P.H) * P.W;
          // weighted gradients of this slice; the segments that use it, listed
          // in ascending order (ballot within a warp, prefix over warps)
          bool any = false;
          if (tid < NSEG) {
            int col = tid % TXB, rb = tid / TXB;
            for (int j = 0; j < SEG; ++j) {
              int yy = ty0 + rb * SEG + j, xx = tx0 + col;
              float2 g = make_float2(0.f, 0.f);
              if (yy < P.H && xx < P.W) {
                int k0;
                float t;
                select_slice(P, yy, xx, P.depth[((size_t)n * P.H + yy) * P.W + xx], &k0, &t);
                float w = (k0 == key) ? (two ? 1.f - t : 1.f)
                                      : ((two && k0 + 1 == key) ? t : 0.f);
                if (w != 0.f) {
                  g.x = w * goL[(size_t)yy * P.W + xx];
                  g.y = w * goR[(size_t)yy * P.W + xx];
                  any = true;
                }
              }
              G[(rb * SEG + j) * TXB + col] = g;
            }
          }
          const unsigned bal = __ballot_sync(0xffffffffu, any);
          const int rank = __popc(bal & ((1u << (tid & 31)) - 1));
          if (tid < NSEG && (tid & 31) == 0) s_wcnt[tid >> 5] = __popc(bal);
          __syncthreads();
          if (tid == 0) {
            int run = 0;
            for (int w = 0; w < NSEG / 32; ++w) {
              int cnt = s_wcnt[w];
              s_wcnt[w] = run;
              run += cnt;
            }
            s_nseg = run;
          }
          __syncthreads();
          if (any) segs[s_wcnt[tid >> 5] + rank] = tid;
          __syncthreads();
          const int nseg = s_nseg;
#pragma unroll
          for (int s = 0; s < SPT; ++s) {
            int st = tid + s * NT;
            if (st >= nstrip) continue;
            int v = st % ks, u0 = (st / ks) * SEG;
            for (int q = 0; q < nseg; ++q) {
              int sgi = segs[q];
              int col = sgi % TXB, rb = sgi / TXB;
              const float* colp = halo + (rb * SEG + u0) * S + col + v;
              float img[2 * SEG - 1];
#pragma unroll
              for (int i = 0; i < 2 * SEG - 1; ++i) img[i] = colp[i * S];
#pragma unroll
              for (int j = 0; j < SEG; ++j) {
                float2 g = G[(rb * SEG + j) * TXB + col];
#pragma unroll
                for (int uu = 0; uu < SEG; ++uu) {
                  acc[s][uu] = fmaf(g.x, img[j + uu], acc[s][uu]);
                  acc[s][SEG + uu] = fmaf(g.y, img[j + uu], acc[s][SEG + uu]);
                }
              }
            }
          }
        }
      }
  // dKf[u][v] -> B[key][lam][side][ks-1-u][ks-1-v] of this part's slab
  float* out = gbank + ((size_t)part * gridDim.x * P.NL + (size_t)key * P.NL + lam) * 2 * ks2;
#pragma unroll
  for (int s = 0; s < SPT; ++s) {
    int st = tid + s * NT;
    if (st >= nstrip) continue;
    int v = st % ks, u0 = (st / ks) * SEG;
#pragma unroll
    for (int uu = 0; uu < SEG; ++uu) {
      int u = u0 + uu;
      if (u >= ks) continue;
      size_t o = (size_t)(ks - 1 - u) * ks + (ks - 1 - v);
      out[o] = acc[s][uu];
      out[ks2 + o] = acc[s][SEG + uu];
    }
  }
}

// Quadrant bank: grad_bank = for each stored element, the sum over the four
// flip classes (class x: other side, column mirrored; class y: row mirrored)
// and the part slabs of the per-key gradients, in a fixed order
// (deterministic).  n = stored elements, n_kl = stored slices x wavelengths.
__global__ void bank_fold_quadrant(const float* __restrict__ parts_buf, size_t n, int parts,
                                   int n_kl, int ks, float* __restrict__ gbank) {
  const size_t ks2 = (size_t)ks * ks, nv = 4 * n;  // elements of one part slab
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t kl = i / (2 * ks2), rem = i - kl * 2 * ks2;
    const int side = (int)(rem / ks2), e = (int)(rem - side * ks2), a = e / ks, b = e - a * ks;
    float acc = 0.f;
    for (int f = 0; f < 4; ++f) {
      const bool mx = f & 1, my = f & 2;
      const int vs = mx ? 1 - side : side, va = my ? ks - 1 - a : a, vb = mx ? ks - 1 - b : b;
      const size_t vi = (((size_t)f * n_kl + kl) * 2 + vs) * ks2 + (size_t)va * ks + vb;
      for (int q = 0; q < parts; ++q) acc += parts_buf[(size_t)q * nv + vi];
    }
    gbank[i] = acc;
  }
}

// grad_bank = sum of the part slabs, added in part order (deterministic)
__global__ void bank_parts_reduce(const float* __restrict__ parts_buf, size_t n, int parts,
                                  float* __restrict__ gbank) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float a = parts_buf[i];
    for (int q = 1; q < parts; ++q) a += parts_buf[(size_t)q * n + i];
    gbank[i] = a;
  }
}

template <int NT, int SPT, class TI>
sd_status launch_bank_bwd(const RenderParams& P, const float* gout, const unsigned* bm, int words,
                          int ntx, int nty, float* gbank, float* parts_buf, int parts,
                          cudaStream_t s) {
  const int ks = P.ks;
  size_t smem = (size_t)(RT_Y + ks - 1 + SEG) * (TXB + ks - 1) * 4 + (size_t)TXB * RT_Y * 8 +
                (size_t)(TXB * RT_Y / SEG) * 4;
  auto k = render_bwd_bank_kernel<NT, SPT, TI>;
  SD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(n_keys(P), P.NL, parts);
  // a quadrant bank's gradients are per key (flip class) first, then folded
  const bool quad = P.fmode == SD_FIELD_QUADRANT;
  k<<<grid, NT, smem, s>>>(P, gout, bm, words, ntx, nty, parts > 1 || quad ? parts_buf : gbank,
                           parts);
  sd_status st = launch_status();
  if (st != SD_OK) return st;
  if (quad) {
    const size_t n = (size_t)P.FC * P.Z * P.NL * 2 * ks * ks;
    bank_fold_quadrant<<<1024, 256, 0, s>>>(parts_buf, n, parts, P.FC * P.Z * P.NL, ks, gbank);
    return launch_status();
  }
  if (parts == 1) return st;
  size_t n = (size_t)n_keys(P) * P.NL * 2 * ks * ks;
  bank_parts_reduce<<<1024, 256, 0, s>>>(parts_buf, n, parts, gbank);
  return launch_status();
}

template <int TX, int VB, int KSMAX, int SB, class TB>
sd_status launch_img_bwd(RenderParams& P, const float* gout, float* gaif, cudaStream_t s) {
  using SM = BwdImgSmem<TX, VB, SB>;
  P.halo_w = TX + P.ks - 1;
  P.halo_h = RT_Y + P.ks - 1 + SB;
  size_t smem = SM::bytes(P.ks);
  auto k = render_bwd_img_kernel<TX, VB, KSMAX, SB, TB>;
  SD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((P.W + TX - 1) / TX, (P.H + RT_Y - 1) / RT_Y, P.N * P.C);
  k<<<grid, SM::NT, smem, s>>>(P, gout, gaif);
  return launch_status();
}

constexpr size_t SMEM_CAP_B = 227 * 1024;
// The bank gradient splits every slice's tiles over BANK_PARTS blocks when the
// workspace holds that many partial banks (heavy slices otherwise set the
// tail of the launch); fewer parts with a smaller workspace.
constexpr int BANK_PARTS = 2;

inline size_t bitmap_bytes(int N, int tx, int ty, int nkeys) {
  return ((size_t)N * tx * ty * bitmap_words(nkeys) * 4 + 255) & ~(size_t)255;
}
// one partial bank: a slab per key (a quadrant bank's keys carry 4 flip classes)
inline size_t bank_bytes(const RenderParams& P) {
  return (size_t)n_keys(P) * P.NL * 2 * P.ks * P.ks * 4;
}

sd_status setup_bwd(const sd_bank_layout* layout, int N, int C, int H, int W,
                    RenderParams& P) {
  if (N < 0 || C < 1 || H < 0 || W < 0) return SD_ERR_ARG;
  if ((long long)N * C > 65535 || (long long)H * W > (1ll << 31)) return SD_ERR_UNSUPPORTED;
  std::memset(&P, 0, sizeof P);
  sd_status st = check_layout(layout, P);
  if (st != SD_OK) return st;
  if (layout->dtype != SD_F32 && layout->dtype != SD_BF16 && layout->dtype != SD_F16)
    return SD_ERR_UNSUPPORTED;
  if (!(P.NL == C || P.NL == 1)) return SD_ERR_ARG;
  if ((long long)n_keys(P) > 65000) return SD_ERR_UNSUPPORTED;
  P.N = N;
  P.C = C;
  P.H = H;
  P.W = W;
  return SD_OK;
}

// 8-pixel segments: 16-pixel segments halve the shared atomics per FMA but
// need ~240 registers (8 warps per SM) and measured slower
template <class TB>
sd_status launch_img_bwd_any(RenderParams& P, const float* gout, float* gaif, cudaStream_t s) {
  // one kernel column per fetch up to ks = 65 (as in the forward: 2.5 %
  // faster with an FP32 bank, 9 % with a BF16 bank, than four columns)
  if (P.ks <= 65 && BwdImgSmem<128, 1, 8>::bytes(P.ks) <= SMEM_CAP_B)
    return launch_img_bwd<128, 1, 65, 8, TB>(P, gout, gaif, s);
  if (BwdImgSmem<64, 4, 8>::bytes(P.ks) <= SMEM_CAP_B)
    return launch_img_bwd<64, 4, 127, 8, TB>(P, gout, gaif, s);
  return launch_img_bwd<64, 2, 127, 8, TB>(P, gout, gaif, s);
}

template <class TI>
sd_status launch_bank_bwd_any(const RenderParams& P, const float* gout, const unsigned* bm,
                              int words, int tx, int ty, float* gbank, float* parts_buf,
                              int parts, cudaStream_t s) {
  int KU = (P.ks + SEG - 1) / SEG * SEG;
  int nstrip = P.ks * (KU / SEG);
  // one strip per thread where the strips fill 512-608 threads (ks = 61..65:
  // 6.76 -> 6.51 ms at 1024x1024x3 against 256 threads x 3 strips, of
  // which a quarter of the slots idle)
  if (nstrip > 512 && nstrip <= 608)
    return launch_bank_bwd<608, 1, TI>(P, gout, bm, words, tx, ty, gbank, parts_buf, parts, s);
  if (nstrip <= 256 * 3)
    return launch_bank_bwd<256, 3, TI>(P, gout, bm, words, tx, ty, gbank, parts_buf, parts, s);
  return launch_bank_bwd<512, 4, TI>(P, gout, bm, words, tx, ty, gbank, parts_buf, parts, s);
}


// ---------------------------------------------------------------------------
// 4. bank gradient on the tensor cores (BF16 image; the weighted gradients
// w * G rounded to BF16; FP32 accumulation in tensor memory)
//
// Block (slice key, wavelength, part) as in pass 3.  For a tile pixel row y
// and a group of 16 kernel rows u0..u0+15 the slice gradient is one product
//   D[(g, r), (side, i)] += sum_x Ipad(y + u0 + g, x0 + 8r + x) Gw_side(y, x - i)
// = dKf_side[u0 + g][8r + i]: M = 128 = 16 kernel rows x 8 column groups,
// N = 32 = 2 sides x 16 shifts, K = the tile's 64 columns + 16.  The A
// operand is the staged image tile read as a Hankel matrix directly from
// its BF16 rows (core-matrix rows 16 bytes apart = 8 columns, K blocks 16
// bytes apart, row groups one image row apart), so no shifted copies of the
// image exist; B is the weighted gradient row at 16 shifts, built per row.
// All kernel-row groups accumulate over every row and tile the block visits
// (160 tensor-memory columns at ks = 65); the epilogue writes each element
// once.  Deterministic (fixed MMA order).
// ---------------------------------------------------------------------------
constexpr int BG_NT = 256;
constexpr int BG_KX = TXB + 16;              // K extent: tile columns + 16 shifts
constexpr int BG_IW = BG_KX + 56;            // staged image columns (8 column groups)
constexpr int BG_IWB = BG_IW * 2;            // its row stride in bytes (272)
constexpr int BG_GW = 8 * 12;                // gradient row: 16 zeros, 64 values, 16 zeros
constexpr int BG_N = 32;
constexpr int BG_KB = BG_KX / 8;             // 10 K blocks
constexpr uint32_t BG_LBO_B = BG_N * 16 + 16;  // B K-block stride, padded: conflict-free builds
constexpr uint32_t BG_BBUF = BG_KB * BG_LBO_B;
constexpr int BG_NB = 4;                     // B ring = producer warps 4..7
constexpr int BG_MAXUG = 5;                  // kernel-row groups (ks <= 80)
constexpr uint32_t BG_WAIT = 1u << 22;

__host__ __device__ inline int bg_nug(int ks) { return (ks + 15) / 16; }
__host__ __device__ inline size_t bg_img_bytes(int ks) {
  return ((size_t)(RT_Y + 16 * bg_nug(ks)) * BG_IWB + 127) / 128 * 128;
}
__host__ __device__ inline size_t bg_smem(int ks) {
  return bg_img_bytes(ks) + (size_t)2 * RT_Y * BG_GW * 2 + (size_t)BG_NB * BG_BBUF;
}

__device__ __forceinline__ bool bg_wait(uint64_t* bar, uint32_t parity, int* err) {
  if (tc::mbar_wait(bar, parity, BG_WAIT, err)) return true;
  atomicExch(err, 1);
  return false;
}

__global__ void __launch_bounds__(BG_NT, 2) bank_grad_tc_kernel(
    const RenderParams P, const float* __restrict__ gout, const unsigned* __restrict__ bm,
    int words, int ntx, int nty, float* __restrict__ gbank, int parts, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_full[BG_NB], s_empty[BG_NB], s_tile, s_done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_rows[RT_Y], s_nrow, s_init;
  __shared__ unsigned s_use;
  const int ks = P.ks, p = (ks - 1) >> 1, nug = bg_nug(ks), rows_st = RT_Y + 16 * nug;
  unsigned char* img = smem;                                       // [rows_st][BG_IW] bf16
  unsigned short* gw = reinterpret_cast<unsigned short*>(smem + bg_img_bytes(ks));  // [2][32][96]
  unsigned char* bring = smem + bg_img_bytes(ks) + (size_t)2 * RT_Y * BG_GW * 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int key = blockIdx.x, lam = blockIdx.y, part = blockIdx.z;
  const bool two = P.Z > 1;
  const int kw = key >> 5;
  const unsigned kbit = 1u << (key & 31);
  const int c_lo = (P.NL == P.C) ? lam : 0, c_hi = (P.NL == P.C) ? lam + 1 : P.C;

  // the gradient rows' zero borders (columns j < 16 and j >= 80) once
  for (int i = tid; i < 2 * RT_Y * 32; i += BG_NT) {
    const int row = i >> 5, jj = i & 31;
    gw[row * BG_GW + (jj < 16 ? jj : 64 + jj)] = 0;
  }
  if (warp == 0) tc::tmem_alloc(&s_tmem, 256);
  if (tid == 0) {
    for (int b = 0; b < BG_NB; ++b) {
      tc::mbar_init(&s_full[b], 32);
      tc::mbar_init(&s_empty[b], 1);
    }
    tc::mbar_init(&s_tile, 1);
    tc::mbar_init(&s_done, 1);
    s_init = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = tc::idesc_bf16_f32(128, BG_N);
  const uint32_t img_a = tc::smem_u32(img), ring_a = tc::smem_u32(bring);
  int c_row = 0, visits = 0;
  unsigned inited = 0;  // kernel-row groups written (MMA thread)

  // the tiles of this part that use the slice, in ascending order
  __shared__ int s_list[BG_NT], s_twc[BG_NT / 32];
  const size_t ntiles = (size_t)P.N * nty * ntx;
  for (size_t t0 = 0; t0 < ntiles; t0 += BG_NT)
    for (int li = 0, nlist = slice_tiles<BG_NT>(bm, words, kw, kbit, t0, ntiles, parts, part,
                                                s_list, s_twc);
         li < nlist; ++li) {
        const size_t tile = t0 + s_list[li];
        const int n = (int)(tile / ((size_t)nty * ntx));
        const int rem = (int)(tile - (size_t)n * nty * ntx);
        const int ty = rem / ntx, tx = rem - ty * ntx;
        const int x0 = tx * TXB, y0 = ty * RT_Y;
        for (int c = c_lo; c < c_hi; ++c, ++visits) {
          // the previous visit's MMAs have read the image, the gradients and
          // their B rows; every producer has finished its builds
          if (visits > 0) {
            if (lane == 0) bg_wait(&s_tile, (uint32_t)(visits - 1) & 1u, err);
            __syncwarp();
          }
          if (tid == 0) s_use = 0u;
          __syncthreads();
          const unsigned short* im =
              reinterpret_cast<const unsigned short*>(P.aif) + ((size_t)n * P.C + c) * P.H * P.W;
          // 8 columns (16 bytes) per item: one vector load inside the image
          // when aligned, clamped scalar loads at the edges.  A thread loads
          // four items before storing them (their latencies overlap).
          constexpr int BG_IPR = 4;  // items per thread and round
          const int nimg = rows_st * (BG_IW / 8);
          for (int i0 = 0; i0 < nimg; i0 += BG_IPR * BG_NT) {
            uint4 iv[BG_IPR];
#pragma unroll
            for (int t = 0; t < BG_IPR; ++t) {
              const int i = i0 + tid + t * BG_NT;
              iv[t] = make_uint4(0u, 0u, 0u, 0u);
              if (i < nimg) {
                const int r = i / (BG_IW / 8), q = i - r * (BG_IW / 8);
                const size_t ro = (size_t)min(max(y0 + r - p, 0), P.H - 1) * P.W;
                const int xa = x0 - p + 8 * q;
                const unsigned short* src = im + ro + xa;
                if (xa >= 0 && xa + 8 <= P.W && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                  iv[t] = __ldg(reinterpret_cast<const uint4*>(src));
                } else {
                  uint32_t e[8];
#pragma unroll
                  for (int k = 0; k < 8; ++k) e[k] = im[ro + min(max(xa + k, 0), P.W - 1)];
                  iv[t] = make_uint4(e[0] | (e[1] << 16), e[2] | (e[3] << 16),
                                     e[4] | (e[5] << 16), e[6] | (e[7] << 16));
                }
              }
            }
#pragma unroll
            for (int t = 0; t < BG_IPR; ++t) {
              const int i = i0 + tid + t * BG_NT;
              if (i < nimg) {
                const int r = i / (BG_IW / 8), q = i - r * (BG_IW / 8);
                *reinterpret_cast<uint4*>(img + (size_t)r * BG_IWB + 16 * q) = iv[t];
              }
            }
          }
          // the tile's 2048 pixels, 8 per thread in two rounds of 4: depths and
          // output gradients loaded first, then the selection and the
          // weighted BF16 values
          const float* goL = gout + (((size_t)n * 2 * P.C + c) * P.H) * P.W;
          const float* goR = gout + (((size_t)n * 2 * P.C + P.C + c) * P.H) * P.W;
          constexpr int BG_PPR = 4;
          for (int t0 = 0; t0 < RT_Y * TXB / BG_NT; t0 += BG_PPR) {
            float dq[BG_PPR], gq[BG_PPR][2];
#pragma unroll
            for (int t = 0; t < BG_PPR; ++t) {
              const int i = tid + (t0 + t) * BG_NT, r = i / TXB, x = i - r * TXB;
              const int yy = y0 + r, xx = x0 + x;
              const bool in = yy < P.H && xx < P.W;
              const size_t o = (size_t)yy * P.W + xx;
              dq[t] = in ? P.depth[(size_t)n * P.H * P.W + o] : 1.f;
              gq[t][0] = in ? goL[o] : 0.f;
              gq[t][1] = in ? goR[o] : 0.f;
            }
#pragma unroll
            for (int t = 0; t < BG_PPR; ++t) {
              const int i = tid + (t0 + t) * BG_NT, r = i / TXB, x = i - r * TXB;
              const int yy = y0 + r, xx = x0 + x;
              float gl = 0.f, gr = 0.f;
              if (yy < P.H && xx < P.W) {
                int k0;
                float tt;
                select_slice(P, yy, xx, dq[t], &k0, &tt);
                const float w = (k0 == key) ? (two ? 1.f - tt : 1.f)
                                            : ((two && k0 + 1 == key) ? tt : 0.f);
                gl = w * gq[t][0];
                gr = w * gq[t][1];
              }
              const unsigned short bl = __bfloat16_as_ushort(__float2bfloat16_rn(gl));
              const unsigned short br = __bfloat16_as_ushort(__float2bfloat16_rn(gr));
              gw[r * BG_GW + x + 16] = bl;
              gw[RT_Y * BG_GW + r * BG_GW + x + 16] = br;
              if ((bl | br) & 0x7fffu) atomicOr(&s_use, 1u << r);
            }
          }
          tc::fence_async_smem();  // the staged image, read by the tensor core
          __syncthreads();
          if (tid == 0) {  // the rows with a non-zero weighted gradient
            int k = 0;
            for (int r = 0; r < RT_Y; ++r)
              if (s_use >> r & 1u) s_rows[k++] = r;
            s_nrow = k;
          }
          __syncthreads();
          const int nrow = s_nrow;
          if (warp >= 4) {
            // producer of ring buffer b: the rows k with (c_row + k) % 4 == b.
            // Task t = (K block kb = t % 10, shift half ih, side): the 8 rows
            // (side, 8 ih + i') of K block kb from gradient words q - 1, q
            const int b = warp - 4;
            for (int k = 0; k < nrow; ++k) {
              const int cg = c_row + k;
              if (cg % BG_NB != b) continue;
              if (cg >= BG_NB) {
                if (lane == 0) bg_wait(&s_empty[b], (uint32_t)(cg / BG_NB - 1) & 1u, err);
                __syncwarp();
              }
              const int y = s_rows[k];
              unsigned char* dstb = bring + (size_t)b * BG_BBUF;
              for (int t = lane; t < 2 * 2 * BG_KB; t += 32) {
                const int kb = t % BG_KB, ih = (t / BG_KB) & 1, side = t / (2 * BG_KB);
                const int q = kb + 2 - ih;
                const unsigned short* row = gw + (size_t)side * RT_Y * BG_GW + y * BG_GW;
                const uint4 w0 = *reinterpret_cast<const uint4*>(row + 8 * (q - 1));
                const uint4 w1 = *reinterpret_cast<const uint4*>(row + 8 * q);
                const uint32_t c8[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                unsigned char* d = dstb + (size_t)kb * BG_LBO_B + (size_t)(side * 16 + 8 * ih) * 16;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  uint32_t g4[4];
#pragma unroll
                  for (int kk = 0; kk < 4; ++kk) {
                    if (i & 1)
                      g4[kk] = __funnelshift_r(c8[(7 - i) / 2 + kk], c8[(9 - i) / 2 + kk], 16);
                    else
                      g4[kk] = c8[(8 - i) / 2 + kk];
                  }
                  *reinterpret_cast<uint4*>(d + i * 16) = make_uint4(g4[0], g4[1], g4[2], g4[3]);
                }
              }
              tc::fence_async_smem();
              tc::mbar_arrive(&s_full[b]);
            }
          } else if (warp == 0) {
            if (lane == 0) {
              for (int k = 0; k < nrow; ++k) {
                const int cg = c_row + k, b = cg % BG_NB;
                if (!bg_wait(&s_full[b], (uint32_t)(cg / BG_NB) & 1u, err)) break;
                tc::fence_after_sync();
                const int y = s_rows[k];
                for (int ug = 0; ug < nug; ++ug)
#pragma unroll
                  for (int s = 0; s < BG_KB / 2; ++s) {
                    const uint64_t ad = tc::smem_desc(
                        img_a + (uint32_t)(y + 16 * ug) * BG_IWB + (uint32_t)s * 32u, 16, BG_IWB);
                    const uint64_t bd = tc::smem_desc(
                        ring_a + (uint32_t)b * BG_BBUF + (uint32_t)s * 2u * BG_LBO_B, BG_LBO_B, 128);
                    tc::mma_bf16(tmem + (uint32_t)(ug * BG_N), ad, bd, idesc,
                                 ((inited >> ug) & 1u) || s > 0);
                    inited |= 1u << ug;
                  }
                tc::commit(&s_empty[b]);
              }
              tc::commit(&s_tile);
            }
            __syncwarp();
          }
          c_row += nrow;
        }
      }
  // every MMA has completed; the accumulator holds the block's gradient
  if (tid == 0) {
    tc::commit(&s_done);
    s_init = (int)inited;
  }
  if (lane == 0) bg_wait(&s_done, 0, err);
  __syncwarp();
  __syncthreads();
  tc::fence_after_sync();
  float* out = gbank + ((size_t)part * gridDim.x * P.NL + (size_t)key * P.NL + lam) * 2 * ks * ks;
  if (warp < 4) {
    const int m = 32 * warp + lane, g = m >> 3, r = m & 7;
    const unsigned ini = (unsigned)s_init;
    for (int ug = 0; ug < nug; ++ug) {
      float v[32];
      tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(ug * BG_N), v);
      const int u = 16 * ug + g;
      if (u >= ks) continue;
#pragma unroll
      for (int side = 0; side < 2; ++side)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          if (i == 8 && r != 7) continue;  // column 64 comes from group 7, shift 8
          const int vv = 8 * r + i;
          if (vv < ks)
            out[(size_t)side * ks * ks + (size_t)(ks - 1 - u) * ks + (ks - 1 - vv)] =
                ((ini >> ug) & 1u) ? v[side * 16 + i] : 0.f;
        }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 256);
}

sd_status launch_bank_grad_tc(const RenderParams& P, const float* gout, const unsigned* bm,
                              int words, int ntx, int nty, float* gbank, float* parts_buf,
                              int parts, int* err, cudaStream_t s) {
  const int ks = P.ks;
  // at least 80 KB: two CTAs per SM, the tensor memory's 512 columns
  const size_t smem = std::max(bg_smem(ks), (size_t)80 * 1024);
  SD_CUDA_TRY(cudaFuncSetAttribute(bank_grad_tc_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const bool quad = P.fmode == SD_FIELD_QUADRANT;
  dim3 grid(n_keys(P), P.NL, parts);
  bank_grad_tc_kernel<<<grid, BG_NT, smem, s>>>(P, gout, bm, words, ntx, nty,
                                                parts > 1 || quad ? parts_buf : gbank, parts, err);
  sd_status st = launch_status();
  if (st != SD_OK) return st;
  if (quad) {
    const size_t n = (size_t)P.FC * P.Z * P.NL * 2 * ks * ks;
    bank_fold_quadrant<<<1024, 256, 0, s>>>(parts_buf, n, parts, P.FC * P.Z * P.NL, ks, gbank);
    return launch_status();
  }
  if (parts == 1) return SD_OK;
  const size_t n = (size_t)n_keys(P) * P.NL * 2 * ks * ks;
  bank_parts_reduce<<<1024, 256, 0, s>>>(parts_buf, n, parts, gbank);
  return launch_status();
}

}  // namespace sd

extern "C" {

sd_status sd_dp_render_backward_workspace(const sd_bank_layout* layout, int N, int C,
                                          int H, int W, size_t* bytes) {
  using namespace sd;
  if (!bytes) return SD_ERR_ARG;
  RenderParams P;
  sd_status st = setup_bwd(layout, N, C, H, W, P);
  if (st != SD_OK) return st;
  int tx, ty;
  bwd_tiles(H, W, &tx, &ty);
  *bytes = bitmap_bytes(N, tx, ty, n_keys(P)) + (size_t)BANK_PARTS * bank_bytes(P);
  return SD_OK;
}

sd_status sd_dp_render_backward(const float* grad_out, const void* aif, const float* depth_m,
                                const void* bank, const sd_bank_layout* layout, int N, int C,
                                int H, int W, int image_dtype, float* grad_aif,
                                float* grad_bank, void* workspace, size_t workspace_bytes,
                                void* stream) {
  using namespace sd;
  if (!grad_out || !aif || !depth_m || !bank) return SD_ERR_ARG;
  if (image_dtype != SD_F32 && image_dtype != SD_BF16 && image_dtype != SD_F16)
    return SD_ERR_UNSUPPORTED;
  RenderParams P;
  sd_status st = setup_bwd(layout, N, C, H, W, P);
  if (st != SD_OK) return st;
  P.aif = aif;
  P.depth = depth_m;
  P.bank = bank;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  size_t bank_elems = (size_t)P.FC * P.Z * P.NL * 2 * P.ks * P.ks;  // stored bank
  if (N == 0 || H == 0 || W == 0) {
    if (grad_bank) SD_CUDA_TRY(cudaMemsetAsync(grad_bank, 0, bank_elems * 4, s));
    return SD_OK;
  }
  if (grad_aif) {
    SD_CUDA_TRY(cudaMemsetAsync(grad_aif, 0, (size_t)N * C * H * W * 4, s));
    // the image pass reads the bank in its storage type
    const int bt = layout->dtype;
    sd_status r = bt == SD_F32    ? launch_img_bwd_any<float>(P, grad_out, grad_aif, s)
                  : bt == SD_BF16 ? launch_img_bwd_any<__nv_bfloat16>(P, grad_out, grad_aif, s)
                                  : launch_img_bwd_any<__half>(P, grad_out, grad_aif, s);
    if (r != SD_OK) return r;
  }
  if (grad_bank) {
    int tx, ty;
    bwd_tiles(H, W, &tx, &ty);
    size_t words = bitmap_words(n_keys(P));
    size_t need = bitmap_bytes(N, tx, ty, n_keys(P));
    // a quadrant bank needs at least one partial bank to fold
    const size_t need_min = need + (P.fmode == SD_FIELD_QUADRANT ? bank_bytes(P) : 0);
    if (!workspace || workspace_bytes < need_min) return SD_ERR_ARG;
    unsigned* bm = reinterpret_cast<unsigned*>(workspace);
    int parts = 1;
    for (int q = BANK_PARTS; q > 1; q >>= 1)
      if (workspace_bytes >= need + (size_t)q * bank_bytes(P)) {
        parts = q;
        break;
      }
    float* parts_buf = reinterpret_cast<float*>(reinterpret_cast<char*>(workspace) + need);
    dim3 g1(tx, ty, N);
    slice_bitmap_kernel<<<g1, NT_BM, words * 4, s>>>(P, bm, (int)words);
    sd_status r = launch_status();
    if (r != SD_OK) return r;
    // the bank pass reads the image in its storage type
    r = image_dtype == SD_F32
            ? launch_bank_bwd_any<float>(P, grad_out, bm, (int)words, tx, ty, grad_bank,
                                         parts_buf, parts, s)
        : image_dtype == SD_BF16
            ? launch_bank_bwd_any<__nv_bfloat16>(P, grad_out, bm, (int)words, tx, ty,
                                                 grad_bank, parts_buf, parts, s)
            : launch_bank_bwd_any<__half>(P, grad_out, bm, (int)words, tx, ty, grad_bank,
                                          parts_buf, parts, s);
    if (r != SD_OK) return r;
  }
  return SD_OK;
}

sd_status sd_dp_render_bank_grad_tc_workspace(const sd_bank_layout* layout, int N, int C,
                                              int H, int W, size_t* bytes) {
  using namespace sd;
  if (!bytes) return SD_ERR_ARG;
  RenderParams P;
  sd_status st = setup_bwd(layout, N, C, H, W, P);
  if (st != SD_OK) return st;
  int tx, ty;
  bwd_tiles(H, W, &tx, &ty);
  *bytes = 256 + bitmap_bytes(N, tx, ty, n_keys(P)) + (size_t)BANK_PARTS * bank_bytes(P);
  return SD_OK;
}

sd_status sd_dp_render_bank_grad_tc(const float* grad_out, const void* aif, const float* depth_m,
                                    const sd_bank_layout* layout, int N, int C, int H, int W,
                                    float* grad_bank, void* workspace, size_t workspace_bytes,
                                    void* stream) {
  using namespace sd;
  if (!grad_out || !aif || !depth_m || !grad_bank) return SD_ERR_ARG;
  RenderParams P;
  sd_status st = setup_bwd(layout, N, C, H, W, P);
  if (st != SD_OK) return st;
  if (P.ks > 16 * BG_MAXUG || bg_smem(P.ks) > 227 * 1024) return SD_ERR_UNSUPPORTED;
  P.aif = aif;
  P.depth = depth_m;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t bank_elems = (size_t)P.FC * P.Z * P.NL * 2 * P.ks * P.ks;
  int tx, ty;
  bwd_tiles(H, W, &tx, &ty);
  const size_t words = bitmap_words(n_keys(P));
  const size_t need = 256 + bitmap_bytes(N, tx, ty, n_keys(P));
  const size_t need_min = need + (P.fmode == SD_FIELD_QUADRANT ? bank_bytes(P) : 0);
  if (!workspace || workspace_bytes < need_min || (reinterpret_cast<uintptr_t>(workspace) & 255))
    return SD_ERR_ARG;
  int* err = reinterpret_cast<int*>(workspace);
  SD_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  if (N == 0 || H == 0 || W == 0) {
    SD_CUDA_TRY(cudaMemsetAsync(grad_bank, 0, bank_elems * 4, s));
    return SD_OK;
  }
  unsigned* bm = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(workspace) + 256);
  int parts = 1;
  for (int q = BANK_PARTS; q > 1; q >>= 1)
    if (workspace_bytes >= need + (size_t)q * bank_bytes(P)) {
      parts = q;
      break;
    }
  float* parts_buf = reinterpret_cast<float*>(reinterpret_cast<char*>(workspace) + need);
  dim3 g1(tx, ty, N);
  slice_bitmap_kernel<<<g1, NT_BM, words * 4, s>>>(P, bm, (int)words);
  st = launch_status();
  if (st != SD_OK) return st;
  return launch_bank_grad_tc(P, grad_out, bm, (int)words, tx, ty, grad_bank, parts_buf, parts,
                             err, s);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Render backward for callers that cannot allocate device memory (for
// example code running where cudaMalloc is forbidden or unavailable: inside
// another framework's allocator-managed region, or a plugin that may only
// use the buffers it is handed).  The bank-gradient pass needs a per-tile
// slice bitmap; here it lives in a fixed device array of this library.
// ---------------------------------------------------------------------------
namespace sd {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;  // 16 MiB per device
static __device__ __align__(256) unsigned g_noalloc_scratch[NOALLOC_SCRATCH_BYTES / 4];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64];  // device address of g_noalloc_scratch, per device

// Device address of the scratch array on the current device; the first call
// on a device looks it up (host code cannot use the array's name as a
// device pointer).
sd_status noalloc_scratch(void** ptr) {
  int dev = 0;
  SD_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return SD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    SD_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *ptr = g_noalloc_ptr[dev];
  return SD_OK;
}

}  // namespace sd

extern "C" sd_status sd_dp_render_backward_noalloc(const float* grad_out, const float* aif,
                                                   const float* depth_m, const float* bank,
                                                   const sd_bank_layout* layout, int N, int C,
                                                   int H, int W, float* grad_aif,
                                                   float* grad_bank, void* stream) {
  using namespace sd;
  void* ws = nullptr;
  size_t need = 0;
  if (grad_bank) {
    // the bitmap must fit; partial banks are used as far as the array allows
    RenderParams P;
    sd_status st = setup_bwd(layout, N, C, H, W, P);
    if (st != SD_OK) return st;
    int tx, ty;
    bwd_tiles(H, W, &tx, &ty);
    need = bitmap_bytes(N, tx, ty, n_keys(P)) +
           (P.fmode == SD_FIELD_QUADRANT ? bank_bytes(P) : 0);
    if (need > NOALLOC_SCRATCH_BYTES) return SD_ERR_CAPACITY;
    st = noalloc_scratch(&ws);
    if (st != SD_OK) return st;
  }
  return sd_dp_render_backward(grad_out, aif, depth_m, bank, layout, N, C, H, W, SD_F32,
                               grad_aif, grad_bank, ws, NOALLOC_SCRATCH_BYTES, stream);
}
