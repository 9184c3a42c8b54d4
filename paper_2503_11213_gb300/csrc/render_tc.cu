// Per-pixel DP render (supplement, "Local DP PSF convolution") of BF16
// images through a BF16 bank on the 5th-generation tensor cores (tcgen05),
// FP32 accumulation in tensor memory.
//
// A CTA renders a tile of 32 rows x 4 columns = 128 pixels (the MMA's M) of
// one channel.  For kernel row u the tile's outputs are a product
//   D[(g, i), n] += sum_v Ipad[y0+g+u, x0+i+v] * Kf_n[u][v],
// rows (g, i) = pixel (tile row g, column i), columns n = (side, slice slot)
// of the up to 8 bank slices the tile's pixels use (N = 16), K = v.  The
// A operand is the image tile staged once in shared memory in the
// no-swizzle K-major core-matrix layout, each image row as 4 consecutive
// 16-byte rows (its 4 column shifts i), so that the operand of kernel row
// u is the same buffer with its descriptor start moved by u image rows; the
// B operand of each kernel row comes from a BF16 copy of the bank re-laid
// out once per call (flipped, rows padded to a multiple of 16) and is
// copied asynchronously (cp.async) into a ring of four shared buffers, 4
// kernel rows at a time, two chunks ahead of the tensor core.  One thread issues the MMAs;
// an mbarrier per buffer reports their completion.  The epilogue reads each
// pixel's row of D from tensor memory and blends its two slices with the
// depth weight.  Tiles using more than 8 slices run one pass per 8.  Two
// CTAs share an SM (about 103 KB of shared memory each at ks = 65), so one
// stages its tile while the other's MMAs run.
//
// Also a device check of the building blocks: one CTA computes D = A_u B^T
// for a 128-row window (starting at row u) of a K-major BF16 matrix, K = 32
// in two MMAs, D in tensor memory.

#include <cuda_bf16.h>

#include "render_common.cuh"
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

// ---------------------------------------------------------------------------
// BF16 render
// ---------------------------------------------------------------------------
constexpr int TR_Y = 32, TR_X = 4, TR_M = 128, TR_NT = 256, TR_N = 16, TR_UC = 4, TR_NB = 4;
constexpr int TR_NPROD = TR_NT - 32;  // producer threads (warps 1..7)
constexpr int TR_GPT = 3;  // B granules per producer per chunk (TR_UC * KB * TR_N <= 640)
constexpr int TR_MAXK = 2 * TR_M;   // candidate slices of a tile (2 per pixel)
constexpr int TR_SI = 4;            // staged (row, K block) items per thread
constexpr int TR_WIN = 4096;        // slice keys of a tile as bits above its smallest
constexpr uint32_t TR_WAIT = 1u << 20;  // completion polls before giving up

__host__ __device__ inline int tr_kp(int ks) { return (ks + 15) / 16 * 16; }
// A: KB K-blocks of R image rows x TR_X shifts x 16 B; B: TR_NB buffers of
// TR_UC kernel rows x KB K-blocks x N rows x 16 B
// K-block stride of the staged A operand: 16 bytes more than the block, so
// that the staging stores of consecutive K blocks fall into different banks
__host__ __device__ inline uint32_t tr_lbo_a(int ks) { return (uint32_t)(TR_Y + ks - 1) * TR_X * 16u + 16u; }
__host__ __device__ inline size_t tr_smem(int ks) {
  const int KP = tr_kp(ks), KB = KP / 8;
  return (size_t)KB * tr_lbo_a(ks) + (size_t)TR_NB * TR_UC * KB * TR_N * 16;
}
inline size_t tr_bp_bytes(const RenderParams& P) {
  return (size_t)P.F * P.Z * P.NL * P.ks * 2 * tr_kp(P.ks) * 2;
}

// bp[key][lam][u][side][v] = bank[key][lam][side][ks-1-u][ks-1-v] (v < ks),
// 0 for ks <= v < KP
template <class TB>
__global__ void tr_bank_kernel(const TB* __restrict__ bank, __nv_bfloat16* __restrict__ bp,
                               size_t n_kl, int ks, int KP) {
  const size_t total = n_kl * ks * 2 * KP;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int v = (int)(i % KP);
    size_t r = i / KP;
    const int side = (int)(r % 2);
    r /= 2;
    const int u = (int)(r % ks);
    const size_t kl = r / ks;
    float val = 0.f;
    if (v < ks)
      val = to_f32<TB>(bank[((kl * 2 + side) * ks + (ks - 1 - u)) * ks + (ks - 1 - v)]);
    bp[i] = __float2bfloat16_rn(val);
  }
}

// Bounded completion wait; a wait that gives up raises the launch's error
// flag at once, which makes every other wait of the launch give up too.
__device__ __forceinline__ bool wait_flag(uint64_t* bar, uint32_t parity, int* err) {
  if (tc::mbar_wait(bar, parity, TR_WAIT, err)) return true;
  atomicExch(err, 1);
  return false;
}

// 16-byte asynchronous global -> shared copy; bytes = 0 writes zeros
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

__global__ void __launch_bounds__(TR_NT, 2) render_tc_kernel(const RenderParams P,
                                                             const __nv_bfloat16* __restrict__ bp,
                                                             int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_cand[TR_MAXK], s_uniq[TR_MAXK], s_wcnt[TR_NT / 32], s_nuniq;
  __shared__ unsigned s_bits[TR_WIN / 32];
  __shared__ int s_wpre[TR_WIN / 32], s_kmin, s_over;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_full[TR_NB], s_empty[TR_NB], s_acc;
  __shared__ long long s_rowb[8];
  const int ks = P.ks, p = (ks - 1) >> 1, KP = tr_kp(ks), KB = KP / 8, R = TR_Y + ks - 1;
  const uint32_t LBO_A = tr_lbo_a(ks), USTR = (uint32_t)KB * TR_N * 16u;
  unsigned char* Asm = smem;
  unsigned char* Bsm = smem + (size_t)KB * LBO_A;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * TR_X, y0 = blockIdx.y * TR_Y;
  const int n = blockIdx.z / P.C, c = blockIdx.z - n * P.C;
  const int lam = (P.NL == P.C) ? c : 0;
  const int H = P.H, W = P.W;
  const bool two = P.Z > 1;

  for (int i = tid; i < TR_WIN / 32; i += TR_NT) s_bits[i] = 0u;
  if (tid == 0) {
    s_kmin = 0x7fffffff;
    s_over = 0;
  }
  __syncthreads();
  // 1. threads 0..127: pixel m = tid (tensor-memory lane m) = tile row m / 4,
  // column m % 4.  Its depth is loaded first and used after the staging
  // loads below have been issued.
  const bool pix = tid < TR_M;
  const int yy = y0 + (tid >> 2), xx = x0 + (tid & 3);
  const bool valid = pix && yy < H && xx < W;
  const float dep = valid ? P.depth[((size_t)n * H + yy) * W + xx] : 1.f;

  // 2. stage the image tile: 16-byte row (image row r, shift i) of K block
  // kb holds Ipad[y0 + r][x0 + i + 8 kb + e], e = 0..7.  Every thread first
  // loads the 12 image values of each of its (row, K block) items (packed in
  // pairs), then builds and stores the 4 shifted rows of each.
  const unsigned short* img =
      reinterpret_cast<const unsigned short*>(P.aif) + ((size_t)n * P.C + c) * H * W;
  const int nitem = R * KB;  // <= TR_SI * TR_NT (checked on the host)
  uint32_t raw[TR_SI][6];
#pragma unroll
  for (int q = 0; q < TR_SI; ++q) {
    const int pr = tid + q * TR_NT;
    if (pr < nitem) {
      const int r = pr / KB, kb = pr - r * KB;
      const size_t rowoff = (size_t)min(max(y0 + r - p, 0), H - 1) * W;
      const int xs = x0 + 8 * kb - p;  // image column of element 0
      const unsigned short* src0 = img + rowoff + xs;
      if (xs >= 0 && xs + TR_X + 8 <= W && (reinterpret_cast<uintptr_t>(src0) & 7) == 0) {
        // interior and the absolute address 8-byte aligned (image planes of
        // an odd size start at odd element offsets): three 8-byte loads
#pragma unroll
        for (int w = 0; w < 3; ++w) {
          const uint2 d = *reinterpret_cast<const uint2*>(src0 + 4 * w);
          raw[q][2 * w] = d.x;
          raw[q][2 * w + 1] = d.y;
        }
      } else {
#pragma unroll
        for (int w = 0; w < 6; ++w) {
          const uint32_t lo = img[rowoff + min(max(xs + 2 * w, 0), W - 1)];
          const uint32_t hi = 2 * w + 1 < TR_X + 7 ? img[rowoff + min(max(xs + 2 * w + 1, 0), W - 1)] : 0u;
          raw[q][w] = lo | (hi << 16);
        }
      }
    }
  }
  int key = -1;
  float t = 0.f;
  if (valid) select_slice(P, yy, xx, dep, &key, &t);
  const bool use0 = valid && (!two || t < 1.f), use1 = valid && two && t > 0.f;
  if (pix) {
    s_cand[2 * tid] = use0 ? key : -1;
    s_cand[2 * tid + 1] = use1 ? key + 1 : -1;
    if (use0 || use1) atomicMin(&s_kmin, use0 ? key : key + 1);
  }
#pragma unroll
  for (int q = 0; q < TR_SI; ++q) {
    const int pr = tid + q * TR_NT;
    if (pr < nitem) {
      const int r = pr / KB, kb = pr - r * KB;
      // element e of the item: half (e & 1) of word e / 2
      auto el = [&](int e) { return (raw[q][e >> 1] >> (16 * (e & 1))) & 0xffffu; };
      unsigned char* dst = Asm + (size_t)kb * LBO_A + (size_t)r * TR_X * 16;
#pragma unroll
      for (int i = 0; i < TR_X; ++i) {
        uint4 w;
        w.x = el(i) | (el(i + 1) << 16);
        w.y = el(i + 2) | (el(i + 3) << 16);
        w.z = el(i + 4) | (el(i + 5) << 16);
        w.w = el(i + 6) | (el(i + 7) << 16);
        *reinterpret_cast<uint4*>(dst + i * 16) = w;
      }
    }
  }
  if (warp == 0) tc::tmem_alloc(&s_tmem, 32);
  if (tid == 0) {
    for (int b = 0; b < TR_NB; ++b) {
      tc::mbar_init(&s_full[b], TR_NPROD);
      tc::mbar_init(&s_empty[b], 1);
    }
    tc::mbar_init(&s_acc, 1);
  }
  tc::fence_async_smem();  // the staged tile, read by the tensor core
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;

  // 3. distinct slices of the tile in ascending order: a bitmap of the
  // candidate keys above the tile's smallest (an exhaustive comparison if a
  // key lies beyond the window), then prefix counts
  const int kmin = s_kmin;
  {
    const int kq = s_cand[tid];
    if (kq >= 0) {
      const int d = kq - kmin;
      if (d < TR_WIN) atomicOr(&s_bits[d >> 5], 1u << (d & 31));
      else s_over = 1;
    }
  }
  __syncthreads();
  const bool over = s_over != 0;
  if (!over) {
    if (warp == 0) {  // exclusive prefix of the bit counts of the words
      int c4[TR_WIN / 32 / 32], tot = 0;
#pragma unroll
      for (int q = 0; q < TR_WIN / 32 / 32; ++q) {
        c4[q] = __popc(s_bits[lane * (TR_WIN / 32 / 32) + q]);
        tot += c4[q];
      }
      int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      int run = incl - tot;
#pragma unroll
      for (int q = 0; q < TR_WIN / 32 / 32; ++q) {
        s_wpre[lane * (TR_WIN / 32 / 32) + q] = run;
        run += c4[q];
      }
      if (lane == 31) s_nuniq = incl;
    }
    __syncthreads();
    for (int w = tid; w < TR_WIN / 32; w += TR_NT) {
      unsigned b = s_bits[w];
      int pos = s_wpre[w];
      while (b) {
        const int bit = __ffs(b) - 1;
        b &= b - 1;
        s_uniq[pos++] = kmin + 32 * w + bit;
      }
    }
  } else {
    const int kq = s_cand[tid];
    bool f = kq >= 0;
    for (int m = 0; m < tid && f; ++m) f = s_cand[m] != kq;
    const int cnt = f ? 1 : 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_wcnt[warp] = incl;
    __syncthreads();
    int base = 0;
    for (int w = 0; w < warp; ++w) base += s_wcnt[w];
    if (f) s_uniq[base + incl - 1] = kq;
    if (tid == TR_NT - 1) s_nuniq = base + incl;
  }
  __syncthreads();
  const int nuniq = s_nuniq;
  auto slot_of = [&](int k) {
    if (!over) {
      const int d = k - kmin;
      return s_wpre[d >> 5] + __popc(s_bits[d >> 5] & ((1u << (d & 31)) - 1u));
    }
    int idx = -1;
    for (int m = 0; m < nuniq; ++m)
      if (s_uniq[m] == k) idx = m;
    return idx;
  };
  const int idx0 = use0 ? slot_of(key) : -1;
  const int idx1 = use1 ? slot_of(key + 1) : -1;
  const float w0 = two ? 1.f - t : 1.f, w1 = t;

  // 4. passes of up to 8 slices.  Warps 1..7 copy the B chunks (TR_UC
  // kernel rows) into a ring of TR_NB buffers with cp.async and report each
  // full buffer on its mbarrier; thread 0 waits for a full buffer, issues
  // its MMAs and lets the tensor core report the buffer empty again, so no
  // CTA barrier sits inside a pass.  At the end of a pass the tensor core
  // reports the accumulator, warps 0..3 fold it into their pixels, and the
  // CTA synchronises before the next pass overwrites it.
  const int nch = (ks + TR_UC - 1) / TR_UC;
  const int npass = (nuniq + 7) / 8;
  const int ngran = TR_UC * KB * TR_N;
  const uint32_t idesc = tc::idesc_bf16_f32(TR_M, TR_N);
  const uint32_t a_base = tc::smem_u32(Asm), b_base = tc::smem_u32(Bsm);
  const uint64_t a_desc0 = tc::smem_desc(a_base, LBO_A, 128);
  const uint64_t b_desc0 = tc::smem_desc(b_base, 256, 128);
  // this producer's granules of a chunk: (kernel row ul, K block kb, column
  // nn), nn fastest; the same for every chunk
  const int ptid = tid - 32;
  uint32_t g_dst[TR_GPT];
  int g_off[TR_GPT], g_ul[TR_GPT], g_sl[TR_GPT];
#pragma unroll
  for (int q = 0; q < TR_GPT; ++q) {
    const int g = ptid + q * TR_NPROD;
    const int nn = g & (TR_N - 1), rest = g >> 4;
    const int kb = rest % KB, ul = rest / KB;
    g_dst[q] = (uint32_t)ul * USTR + kb * 256 + nn * 16;
    g_off[q] = (nn >> 3) * KP + 8 * kb;           // side row, K block
    g_ul[q] = (ptid >= 0 && g < ngran) ? ul : TR_UC;  // TR_UC: no granule
    g_sl[q] = nn & 7;
  }
  float outL = 0.f, outR = 0.f;
  for (int pass = 0; pass < npass; ++pass) {
    if (tid < 8) {  // element offset of each slot's flipped kernel rows
      const int ui = pass * 8 + tid;
      s_rowb[tid] = ui < nuniq ? ((long long)s_uniq[ui] * P.NL + lam) * ks * 2 * KP : -1;
    }
    __syncthreads();
    const int c0 = pass * nch;  // global index of the pass's first chunk
    if (warp == 0) {
      if (lane == 0) {
        for (int ch = 0; ch < nch; ++ch) {
          const int c = c0 + ch, b = c % TR_NB;
          wait_flag(&s_full[b], (uint32_t)(c / TR_NB) & 1u, err);
          tc::fence_after_sync();
          const int urows = min(TR_UC, ks - ch * TR_UC);
          // the start-address field is the low 14 bits (address >> 4)
          uint64_t ad = a_desc0 + (uint64_t)(ch * TR_UC * TR_X);  // rows of 64 B
          uint64_t bd = b_desc0 + (uint64_t)((uint32_t)b * TR_UC * USTR >> 4);
          for (int ul = 0; ul < urows; ++ul) {
            uint64_t a = ad, bb = bd;
            for (int kq = 0; kq < KP / 16; ++kq) {
              tc::mma_bf16(tmem, a, bb, idesc, !(ch == 0 && ul == 0 && kq == 0));
              a += (uint64_t)(2u * LBO_A >> 4);
              bb += (uint64_t)(512u >> 4);
            }
            ad += (uint64_t)TR_X;
            bd += (uint64_t)(USTR >> 4);
          }
          tc::commit(&s_empty[b]);
        }
        tc::commit(&s_acc);
      }
      __syncwarp();
    } else {
      for (int ch = 0; ch < nch; ++ch) {
        const int c = c0 + ch, b = c % TR_NB;
        if (c >= TR_NB)  // the MMAs of chunk c - TR_NB read this buffer
          wait_flag(&s_empty[b], (uint32_t)(c / TR_NB - 1) & 1u, err);
        const uint32_t bdst = b_base + (uint32_t)b * TR_UC * USTR;
#pragma unroll
        for (int q = 0; q < TR_GPT; ++q) {
          const int u = ch * TR_UC + g_ul[q];
          const long long rb = s_rowb[g_sl[q]];
          if (g_ul[q] < TR_UC && u < ks && rb >= 0)
            cp16(bdst + g_dst[q], bp + rb + (long long)u * 2 * KP + g_off[q], 16);
        }
        cp_commit();
        if (ch > 0) {  // the previous chunk has landed: report it
          cp_wait<1>();
          tc::fence_async_smem();
          tc::mbar_arrive(&s_full[(c - 1) % TR_NB]);
        }
      }
      cp_wait<0>();
      tc::fence_async_smem();
      tc::mbar_arrive(&s_full[(c0 + nch - 1) % TR_NB]);
    }
    // the pass's accumulator
    if (warp < TR_M / 32) {
      wait_flag(&s_acc, (uint32_t)pass & 1u, err);
      tc::fence_after_sync();
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16), v);
#pragma unroll
      for (int sl = 0; sl < 8; ++sl) {
        const int ui = pass * 8 + sl;
        if (ui == idx0) {
          outL = fmaf(w0, v[sl], outL);
          outR = fmaf(w0, v[8 + sl], outR);
        }
        if (ui == idx1) {
          outL = fmaf(w1, v[sl], outL);
          outR = fmaf(w1, v[8 + sl], outR);
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (valid) {
    __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(P.out);
    out[(((size_t)n * 2 * P.C + c) * H + yy) * W + xx] = __float2bfloat16_rn(outL);
    out[(((size_t)n * 2 * P.C + P.C + c) * H + yy) * W + xx] = __float2bfloat16_rn(outR);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 32);
}

}  // namespace sd

extern "C" sd_status sd_dp_render_tc_workspace(const sd_bank_layout* layout, size_t* bytes) {
  using namespace sd;
  if (!bytes) return SD_ERR_ARG;
  RenderParams P;
  std::memset(&P, 0, sizeof P);
  sd_status st = check_layout(layout, P);
  if (st != SD_OK) return st;
  *bytes = 256 + tr_bp_bytes(P);
  return SD_OK;
}

extern "C" sd_status sd_dp_render_tc(const void* aif, const float* depth_m, const void* bank,
                                     const sd_bank_layout* layout, int N, int C, int H, int W,
                                     void* out, void* workspace, size_t workspace_bytes,
                                     void* stream) {
  using namespace sd;
  if (!aif || !depth_m || !bank || !out) return SD_ERR_ARG;
  if (N < 0 || C < 1 || H < 0 || W < 0) return SD_ERR_ARG;
  RenderParams P;
  std::memset(&P, 0, sizeof P);
  sd_status st = check_layout(layout, P);
  if (st != SD_OK) return st;
  if (layout->dtype != SD_BF16 && layout->dtype != SD_F32) return SD_ERR_UNSUPPORTED;
  if (P.ks > 65 || tr_smem(P.ks) > 227 * 1024 ||
      (TR_Y + P.ks - 1) * (tr_kp(P.ks) / 8) > TR_SI * TR_NT)
    return SD_ERR_UNSUPPORTED;
  if (!(P.NL == C || P.NL == 1)) return SD_ERR_ARG;
  if ((long long)N * C > 65535 || (long long)H * W > (1ll << 31) ||
      (H + TR_Y - 1) / TR_Y > 65535)
    return SD_ERR_UNSUPPORTED;
  if (!workspace || workspace_bytes < 256 + tr_bp_bytes(P) ||
      (reinterpret_cast<uintptr_t>(workspace) & 255))
    return SD_ERR_ARG;
  if (N == 0 || H == 0 || W == 0) return SD_OK;
  P.aif = aif;
  P.depth = depth_m;
  P.bank = bank;
  P.out = out;
  P.N = N;
  P.C = C;
  P.H = H;
  P.W = W;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* err = reinterpret_cast<int*>(workspace);
  __nv_bfloat16* bp = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(workspace) + 256);
  SD_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  const size_t n_kl = (size_t)P.F * P.Z * P.NL;
  if (layout->dtype == SD_BF16)
    tr_bank_kernel<__nv_bfloat16><<<1024, 256, 0, s>>>(
        reinterpret_cast<const __nv_bfloat16*>(bank), bp, n_kl, P.ks, tr_kp(P.ks));
  else
    tr_bank_kernel<float><<<1024, 256, 0, s>>>(reinterpret_cast<const float*>(bank), bp, n_kl,
                                               P.ks, tr_kp(P.ks));
  st = launch_status();
  if (st != SD_OK) return st;
  const size_t smem = tr_smem(P.ks);
  SD_CUDA_TRY(cudaFuncSetAttribute(render_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  dim3 grid((W + TR_X - 1) / TR_X, (H + TR_Y - 1) / TR_Y, N * C);
  render_tc_kernel<<<grid, TR_NT, smem, s>>>(P, bp, err);
  return launch_status();
}

extern "C" sd_status sd_dev_tc_check(const void* a, const void* b, int u, float* d,
                                     int32_t* status, void* stream) {
  using namespace sd;
  if (!a || !b || !d || !status || u < 0 || u > TCC_ROWS - TCC_M) return SD_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  tc_check_kernel<<<1, 128, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(a),
                                    reinterpret_cast<const __nv_bfloat16*>(b), u, d, status);
  return launch_status();
}
