// Per-pixel DP rendering (supplement, "Local DP PSF convolution") on sm_103a.
//
// out_L[n,c,y,x] = sum_{u,v} Ipad[n,c,y+u,x+v] * K_L(y,x,c)[ks-1-u][ks-1-v]
// with Ipad the image replicate-padded by p = (ks-1)/2 (likewise R) and, in
// bank mode, K(y,x,c) = (1-t) B[f][z0][lam] + t B[f][z0+1][lam] selected per
// pixel from its radial image height and depth (linear in inverse depth);
// with a quadrant bank, from the nearest first-quadrant field point of
// (|X|, |Y|) and the PSF's flip symmetry about both axes (Sec. 5.3).
//
// The render is linear in the kernel, so a pixel's output is
// (1-t) (I * B[f][z0]) + t (I * B[f][z0+1]): a sum over bank slices with
// per-pixel weights.  Neighbouring pixels use different slices (field index
// and depth bracket both vary), so each thread block, for one image tile and
// one channel:
//   1. selects (slice key, t) per pixel in FP32 without contraction;
//   2. splits the tile into vertical segments of SEG pixels and marks, per
//      slice key, the segments that need it (a bitmask per key);
//   3. cuts every key's segment list into chunks of 32 (one lane per
//      segment, lanes in column order so shared-memory reads of the staged
//      tile are conflict-free);
//   4. each warp takes chunks; for a chunk it streams the key's taps
//      through a warp-private shared-memory buffer, VB columns at a time,
//      prefetching the next block into registers while computing, and each
//      lane slides a register window of SEG image rows down the staged
//      tile+halo: per tap one shared load of the image, one broadcast load of
//      the (L, R) tap pair and 2*SEG FMAs;
//   5. weighted segment results go to a shared accumulator.  Every pixel
//      receives at most two non-zero contributions (its two slices), so the
//      order of the additions cannot change the result: deterministic.

#define SD_TU 2  // translation unit id of this file's SD_CHECK sites
#include "render_common.cuh"

namespace sd {

// Shared-memory layout of one block (sizes in 4-byte words).
template <int TX, int VB>
struct RenderSmem {
  static constexpr int NT = 4 * TX;          // threads = segments
  static constexpr int NW = NT / 32;         // warps
  static constexpr int NPX = TX * RT_Y;      // pixels per tile
  static constexpr int MW = NT / 32;         // mask words per key
  // tap rows padded to a multiple of SEG (zeros beyond ks): 2 buffers
  __host__ __device__ static int ku(int ks) { return (ks + SEG - 1) / SEG * SEG; }
  __host__ __device__ static size_t kbuf_words(int ks) { return (size_t)2 * (2 * ku(ks) * VB); }
  __host__ __device__ static size_t halo_words(int ks) { return (size_t)(TX + ks - 1) * (RT_Y + ks - 1 + SEG); }
  static size_t bytes(int ks) {
    size_t w = halo_words(ks) + NW * kbuf_words(ks) + 3 * (size_t)NPX  // halo, K, accL/R, t
               + (size_t)RK * MW + (RK + 1) + MAX_CHUNKS               // masks, prefix, chunks
               + NPX / 2;                                              // u16 keys
    return 4 * w;
  }
};

template <class TB>
__device__ __forceinline__ float ldk(const TB* p) { return to_f32<TB>(__ldg(p)); }

template <class TI, class TB, int TX, int VB, int KSMAX>
__global__ void __launch_bounds__(4 * TX, 1) render_fwd_kernel(const RenderParams P) {
  using SM = RenderSmem<TX, VB>;
  constexpr int NT = SM::NT, NW = SM::NW, NPX = SM::NPX, MW = SM::MW;
  constexpr int NR = (2 * ((KSMAX + SEG - 1) / SEG * SEG) * VB + 31) / 32;  // prefetch regs
  extern __shared__ __align__(16) unsigned char smem[];
  const int ks = P.ks, p = (ks - 1) >> 1, ks2 = ks * ks;
  const int S = P.halo_w;
  float* halo = reinterpret_cast<float*>(smem);
  float* kbuf = halo + SM::halo_words(ks);                   // NW x 2 x [ks][VB][2]
  float* accL = kbuf + NW * SM::kbuf_words(ks);
  float* accR = accL + NPX;
  float* pt = accR + NPX;
  unsigned* mask = reinterpret_cast<unsigned*>(pt + NPX);     // [RK][MW]
  int* kpre = reinterpret_cast<int*>(mask + RK * MW);         // [RK + 1]
  int* chunks = kpre + RK + 1;                                // [MAX_CHUNKS]
  unsigned short* prel = reinterpret_cast<unsigned short*>(chunks + MAX_CHUNKS);
  __shared__ int s_kmin, s_kmax, s_nchunks, s_next;

  const int tx0 = blockIdx.x * TX, ty0 = blockIdx.y * RT_Y;
  const int n = blockIdx.z / P.C, c = blockIdx.z - n * P.C;
  const int lam = (P.NL == P.C) ? c : 0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int H = P.H, W = P.W;
  const bool two = (P.Z > 1);

  // ---- 1. per-pixel selection; stage the tile + halo -------------------------
  const int seg_col = tid % TX, seg_rb = tid / TX;
  int kmin_t = 0x7fffffff, kmax_t = -1;
  int key_j[SEG];
  float t_j[SEG];
#pragma unroll
  for (int j = 0; j < SEG; ++j) {
    int yy = ty0 + seg_rb * SEG + j, xx = tx0 + seg_col;
    key_j[j] = -1;
    t_j[j] = 0.f;
    if (yy < H && xx < W) {
      float d = P.depth[((size_t)n * H + yy) * W + xx];
      select_slice(P, yy, xx, d, &key_j[j], &t_j[j]);
      kmin_t = min(kmin_t, key_j[j]);
      kmax_t = max(kmax_t, key_j[j] + (two ? 1 : 0));
    }
    pt[(seg_rb * SEG + j) * TX + seg_col] = t_j[j];
  }
  if (tid == 0) {
    s_kmin = 0x7fffffff;
    s_kmax = -1;
  }
  // the tile and its halo, one warp per row: 16-byte loads of EPV columns
  // wherever such a group lies inside the image row at a 16-byte aligned
  // address, clamped single loads at the image edges (replicate padding)
  const TI* img = reinterpret_cast<const TI*>(P.aif) + ((size_t)n * P.C + c) * H * W;
  {
    constexpr int EPV = 16 / (int)sizeof(TI);
    const int x_lo = tx0 - p;  // image column of halo column 0
    for (int r = warp; r < P.halo_h; r += NW) {
      const size_t rowoff = (size_t)min(max(ty0 + r - p, 0), H - 1) * W;
      const TI* src = img + rowoff;
      // first column at or left of x_lo whose address is 16-byte aligned
      const int mis = (int)((reinterpret_cast<uintptr_t>(src) / sizeof(TI) + (size_t)(x_lo + 4 * EPV)) % EPV);
      const int xa = x_lo - mis;
      const int ng = (S + mis + EPV - 1) / EPV;
      for (int g = lane; g < ng; g += 32) {
        const int x = xa + g * EPV;
        float v[EPV];
        if (x >= 0 && x + EPV <= W) {
          const uint4 q = __ldg(reinterpret_cast<const uint4*>(src + x));
          const TI* e = reinterpret_cast<const TI*>(&q);
#pragma unroll
          for (int k = 0; k < EPV; ++k) v[k] = to_f32<TI>(e[k]);
        } else {
#pragma unroll
          for (int k = 0; k < EPV; ++k) v[k] = to_f32<TI>(src[min(max(x + k, 0), W - 1)]);
        }
#pragma unroll
        for (int k = 0; k < EPV; ++k) {
          const int cc = x + k - x_lo;
          if (cc >= 0 && cc < S) halo[r * S + cc] = v[k];
        }
      }
    }
  }
  for (int i = tid; i < NPX; i += NT) {
    accL[i] = 0.f;
    accR[i] = 0.f;
  }
  __syncthreads();
  atomicMin(&s_kmin, kmin_t);
  atomicMax(&s_kmax, kmax_t);
  __syncthreads();
  const int kmin = s_kmin, kmax = s_kmax;
#pragma unroll
  for (int j = 0; j < SEG; ++j)
    prel[(seg_rb * SEG + j) * TX + seg_col] =
        (unsigned short)(key_j[j] >= 0 ? key_j[j] - kmin : 0xffff);

  float* kb = kbuf + warp * SM::kbuf_words(ks);  // this warp's 2 x [ks][VB][side]
  const int nblk = (ks + VB - 1) / VB;
  const int KU = SM::ku(ks);
  const int kb_elems = 2 * KU * VB;

  for (int wbase = kmin; wbase <= kmax; wbase += RK) {
    // ---- 2. segment bitmask per key of the window ---------------------------
    for (int i = tid; i < RK * MW; i += NT) mask[i] = 0u;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
      int k0 = key_j[j];
      if (k0 < 0) continue;
      float t = t_j[j];
      // slices with zero weight need no work
      if ((!two || t < 1.f) && k0 >= wbase && k0 < wbase + RK)
        atomicOr(&mask[(k0 - wbase) * MW + warp], 1u << lane);
      if (two && t > 0.f && k0 + 1 >= wbase && k0 + 1 < wbase + RK)
        atomicOr(&mask[(k0 + 1 - wbase) * MW + warp], 1u << lane);
    }
    __syncthreads();
    // ---- 3. chunks of 32 segments per key (warp 0 scans the key counts) -----
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
    const int nchunks = s_nchunks;  // <= NT * 2 * SEG / 32 + RK <= MAX_CHUNKS
    for (int k = tid; k < RK; k += NT)
      for (int q = kpre[k]; q < kpre[k + 1]; ++q) chunks[q] = (k << 8) | (q - kpre[k]);
    if (tid == 0) s_next = NW;
    __syncthreads();

    // ---- 4. warps take chunks (first one by index, then from a counter) -------
    for (int ch = warp; ch < nchunks;) {
      const int rel = chunks[ch] >> 8, sub = chunks[ch] & 0xff;
      const int key = wbase + rel;
      // this lane's segment: the (sub*32 + lane)-th set bit of the key mask
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
      // segment id = warp * 32 + lane of the owner thread = rb * TX + col
      const int col = sg % TX, rb = sg / TX;
      const int f = key / P.Z, z = key - f * P.Z;
      // quadrant bank: field cell and flips (x: mirror columns and exchange
      // L and R; y: mirror rows); radial bank: flips = 0
      const int flips = f / P.FC, cell = f - flips * P.FC;
      const TB* K0 = reinterpret_cast<const TB*>(P.bank) +
                     (((size_t)cell * P.Z + z) * P.NL + lam) * 2 * ks2;
      const TB* KL = (flips & 1) ? K0 + ks2 : K0;
      const TB* KR = (flips & 1) ? K0 : K0 + ks2;
      const bool mx = flips & 1, my = flips & 2;
      // K block b covers v in [b*VB, b*VB + VB): element (u, vv, side) =
      // K_side[ks-1-u][ks-1-(b*VB+vv)] at kb[buf][(u*VB + vv)*2 + side]
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
              v = ldk<TB>((side ? KR : KL) + (my ? u : ks - 1 - u) * ks + (mx ? v_ : ks - 1 - v_));
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
      // rows [ulo, uhi] of the fetched block holding a non-zero tap (of
      // either side): blur discs leave many kernel rows empty
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
      // (L, R) sums of the SEG pixels: one packed two-lane FMA per tap and
      // pixel (its components round like fmaf)
      float2 a2[SEG];
#pragma unroll
      for (int j = 0; j < SEG; ++j) a2[j] = make_float2(0.f, 0.f);
      const float* base = halo + (rb * SEG) * S + col;
      for (int b = 0; b < nblk; ++b) {
        const float* kcur = kb + (b & 1) * kb_elems;
        const int ulo = ulo_n, uhi = uhi_n;
        if (b + 1 < nblk) fetch(b + 1);  // loads in flight during the compute
        // rows u0 in [u_begin, uhi]: the taps outside are zero (KU = ks
        // rounded up to SEG; the padding taps are zero too)
        const int u_begin = (ulo / SEG) * SEG;
        const int vmax = uhi < 0 ? 0 : min(VB, ks - b * VB);
        for (int vv = 0; vv < vmax; ++vv) {
          // the deepest halo row this column's window reaches
          if (!SD_CHECK((size_t)(rb * SEG + (uhi / SEG) * SEG + 2 * SEG - 1) * S + col + b * VB + vv,
                        SM::halo_words(ks)))
            continue;
          const float* colp = base + b * VB + vv;
          float win[SEG];
#pragma unroll
          for (int j = 0; j < SEG; ++j) win[j] = colp[(u_begin + j) * S];
          const float2* kp = reinterpret_cast<const float2*>(kcur) + vv;
          for (int u0 = u_begin; u0 <= uhi; u0 += SEG) {
#pragma unroll
            for (int q = 0; q < SEG; ++q) {
              const int u = u0 + q;
              float2 w2 = kp[u * VB];
#pragma unroll
              for (int j = 0; j < SEG; ++j) {
                const float iv = win[(q + j) % SEG];
                a2[j] = __ffma2_rn(make_float2(iv, iv), w2, a2[j]);
              }
              win[q] = colp[(u + SEG) * S];
            }
          }
        }
        if (b + 1 < nblk) {
          extent(ulo_n, uhi_n);
          commit(kb + ((b + 1) & 1) * kb_elems);
        }
        __syncwarp();
      }
      if (act) {
#pragma unroll
        for (int j = 0; j < SEG; ++j) {
          int pix = (rb * SEG + j) * TX + col;
          if (!SD_CHECK(pix, SM::NPX)) continue;
          unsigned short r16 = prel[pix];
          if (r16 == 0xffff) continue;
          int k0 = kmin + (int)r16;
          float t = pt[pix];
          float w = (k0 == key) ? (two ? 1.f - t : 1.f) : ((two && k0 + 1 == key) ? t : 0.f);
          if (w != 0.f) {
            atomicAdd(&accL[pix], a2[j].x * w);
            atomicAdd(&accR[pix], a2[j].y * w);
          }
        }
      }
      int nxt = 0;
      if (lane == 0) nxt = atomicAdd(&s_next, 1);
      ch = __shfl_sync(0xffffffffu, nxt, 0);
    }
    __syncthreads();
  }
  // ---- 5. write the L and R planes of channel c ---------------------------------
  TI* outL = reinterpret_cast<TI*>(P.out) + (((size_t)n * 2 * P.C + c) * H) * W;
  TI* outR = reinterpret_cast<TI*>(P.out) + (((size_t)n * 2 * P.C + P.C + c) * H) * W;
  for (int i = tid; i < NPX; i += NT) {
    int yy = ty0 + i / TX, xx = tx0 + i % TX;
    if (yy < H && xx < W) {
      outL[(size_t)yy * W + xx] = from_f32<TI>(accL[i]);
      outR[(size_t)yy * W + xx] = from_f32<TI>(accR[i]);
    }
  }
}

template <class TI, class TB, int TX, int VB, int KSMAX>
sd_status launch_fwd_cfg(RenderParams& P, cudaStream_t s) {
  using SM = RenderSmem<TX, VB>;
  P.halo_w = TX + P.ks - 1;
  P.halo_h = RT_Y + P.ks - 1 + SEG;
  size_t smem = SM::bytes(P.ks);
  auto k = render_fwd_kernel<TI, TB, TX, VB, KSMAX>;
  SD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((P.W + TX - 1) / TX, (P.H + RT_Y - 1) / RT_Y, P.N * P.C);
  k<<<grid, SM::NT, smem, s>>>(P);
  return launch_status();
}

constexpr size_t SMEM_CAP = 227 * 1024;

template <class TI, class TB>
sd_status launch_fwd(RenderParams& P, cudaStream_t s) {
  // the widest tile whose block fits in shared memory.  Up to ks = 65 the
  // kernel columns are fetched one at a time: the row extent of non-zero
  // taps is then taken per column (more empty rows skipped) and the smaller
  // tap buffers leave more shared storage to L1; measured 8 % (FP32 bank)
  // to 15 % (BF16 bank) faster at 1024x1024x3 than four columns at a time.
  if (P.ks <= 65 && RenderSmem<128, 1>::bytes(P.ks) <= SMEM_CAP)
    return launch_fwd_cfg<TI, TB, 128, 1, 65>(P, s);
  if (RenderSmem<64, 4>::bytes(P.ks) <= SMEM_CAP) return launch_fwd_cfg<TI, TB, 64, 4, 127>(P, s);
  return launch_fwd_cfg<TI, TB, 64, 2, 127>(P, s);
}

}  // namespace sd

extern "C" {

sd_status sd_dp_render(const void* aif, const float* depth_m, const void* bank,
                       const sd_bank_layout* layout, int N, int C, int H, int W,
                       int image_dtype, void* out, void* stream) {
  SD_API_RANGE("sd_dp_render");
  using namespace sd;
  if (!aif || !depth_m || !bank || !out) return SD_ERR_ARG;
  if (N < 0 || C < 1 || H < 0 || W < 0) return SD_ERR_ARG;
  if (N == 0 || H == 0 || W == 0) return SD_OK;
  if ((long long)N * C > 65535 || (long long)H * W > (1ll << 31)) return SD_ERR_UNSUPPORTED;
  RenderParams P;
  std::memset(&P, 0, sizeof P);
  sd_status st = check_layout(layout, P);
  if (st != SD_OK) return st;
  if (!(P.NL == C || P.NL == 1)) return SD_ERR_ARG;
  // 16-bit relative keys (quadrant keys carry 4 flip classes)
  if ((long long)P.FC * P.Z * (P.fmode == SD_FIELD_QUADRANT ? 4 : 1) > 65000)
    return SD_ERR_UNSUPPORTED;
  P.aif = aif;
  P.depth = depth_m;
  P.bank = bank;
  P.out = out;
  P.N = N;
  P.C = C;
  P.H = H;
  P.W = W;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int bt = layout->dtype;
  if (image_dtype == SD_F32 && bt == SD_F32) return launch_fwd<float, float>(P, s);
  if (image_dtype == SD_F32 && bt == SD_BF16) return launch_fwd<float, __nv_bfloat16>(P, s);
  if (image_dtype == SD_BF16 && bt == SD_BF16)
    return launch_fwd<__nv_bfloat16, __nv_bfloat16>(P, s);
  if (image_dtype == SD_F16 && bt == SD_F16) return launch_fwd<__half, __half>(P, s);
  if (image_dtype == SD_F32 && bt == SD_F16) return launch_fwd<float, __half>(P, s);
  return SD_ERR_UNSUPPORTED;
}

}  // extern "C"

SD_CHECK_TU(render)
