// Per-pixel DP render (supplement, "Local DP PSF convolution") of BF16 or
// FP16 images through a bank in the same type on the 5th-generation tensor
// cores (tcgen05), FP32 accumulation in tensor memory.
//
// A CTA renders a tile of 32 rows x 16 columns of one channel as 4 column
// blocks of 4 pixels.  For kernel row u the tile's outputs are a product
// (M = 128, N = 64, K = the kernel row plus 3, padded to 16):
//   D[(g, cb), (i, side, slot)] += sum_w Ipad[y0+g+u, x0+4cb+w] * Kf[u][w-i]
// rows (g, cb) = tile row g, column block cb; columns = shift i of the
// block's pixel x0+4cb+i, side and one of the up to 8 bank slices the tile
// uses.  A is the image tile staged once in shared memory (no-swizzle
// K-major core matrices, the 4 blocks of an image row as consecutive 16-byte
// rows), so the operand of kernel row u is the same buffer with its
// descriptor start moved by u image rows.  B holds each slice's flipped
// kernel row 4 times, shifted by i = 0..3 (a banded copy), so one image
// operand row serves 4 pixels x 16 (side, slot) columns: the shared-memory
// bytes the tensor core reads per output are a quarter of those of a
// pixels-as-rows product with N = 16.  Four producer warps build the B
// chunks (one kernel row each) from a BF16 re-layout of the bank made once
// per call (flipped, rows padded to a multiple of 16) into a ring of four
// buffers and report them on mbarriers; one thread issues the MMAs and the
// tensor core reports each buffer empty again.  The epilogue reads each
// pixel's 16 columns from tensor memory and blends its two slices with the
// depth weight.  Tiles using more than 8 slices run one pass per 8.  Two
// CTAs share an SM (about 108 KB of shared memory each at ks = 65).
//
// Also a device check of the building blocks: one CTA computes D = A_u B^T
// for a 128-row window (starting at row u) of a K-major BF16 matrix, K = 32
// in two MMAs, D in tensor memory.

#define SD_TU 5  // translation unit id of this file's SD_CHECK sites
#include <algorithm>

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
constexpr int TR_Y = 32;              // tile rows
constexpr int TR_CB = 4;              // column blocks of a tile (A rows per image row)
constexpr int TR_J = 4;               // pixels per column block (shifted copies in B)
constexpr int TR_XW = TR_CB * TR_J;   // tile width
constexpr int TR_M = 128;             // A rows = TR_Y * TR_CB
constexpr int TR_NT = 256;
constexpr int TR_SL = 8;              // slices per pass
constexpr int TR_SS = 2 * TR_SL;      // (side, slot) rows of B per shift
constexpr int TR_N = TR_J * TR_SS;    // 64
constexpr int TR_NB = 4;              // B ring buffers = producer warps 4..7
constexpr int TR_MAXK = 2 * TR_Y * TR_XW;  // candidate slices of a tile (2 per pixel)
constexpr int TR_SI = 4;              // staged (row, K block) items per thread
constexpr int TR_TPL = 5;             // B tasks per producer lane and kernel row (16 KB <= 160)
constexpr int TR_WIN = 4096;          // slice keys of a tile as bits above its smallest
constexpr uint32_t TR_WAIT = 1u << 20;  // completion polls before giving up
constexpr uint32_t TR_DRAIN = 1u << 24;  // final wait for the CTA's own products

// bank rows: flipped kernel rows padded to a multiple of 16 elements
__host__ __device__ inline int tr_kp(int ks) { return (ks + 15) / 16 * 16; }
// K extent of the products: the kernel row plus the TR_J - 1 shifts
__host__ __device__ inline int tr_kk(int ks) { return (ks + TR_J - 1 + 15) / 16 * 16; }
// K-block stride of the staged A operand: 16 bytes more than the block, so
// that the staging stores of consecutive K blocks fall into different banks
__host__ __device__ inline uint32_t tr_lbo_a(int ks) {
  return (uint32_t)(TR_Y + ks - 1) * TR_CB * 16u + 16u;
}
__host__ __device__ inline size_t tr_a_bytes(int ks) {
  return ((size_t)(tr_kk(ks) / 8) * tr_lbo_a(ks) + 1023) / 1024 * 1024;
}
// one B buffer: a kernel row's K blocks of TR_N rows x 16 bytes
__host__ __device__ inline size_t tr_b_bytes(int ks) { return (size_t)(tr_kk(ks) / 8) * TR_N * 16; }
__host__ __device__ inline size_t tr_smem(int ks) {
  return tr_a_bytes(ks) + (size_t)TR_NB * tr_b_bytes(ks);
}
// slices of the re-laid-out bank: every key the selection can produce (a
// quadrant bank's keys carry 4 flip classes)
inline size_t tr_slices(const RenderParams& P) {
  return (size_t)P.FC * P.Z * (P.fmode == SD_FIELD_QUADRANT ? 4 : 1);
}
inline size_t tr_bp_bytes(const RenderParams& P) {
  return tr_slices(P) * P.NL * P.ks * 2 * tr_kp(P.ks) * 2;
}

// bp[key][lam][u][side][v] = bank[key][lam][side][ks-1-u][ks-1-v] (v < ks),
// 0 for ks <= v < KP.  Quadrant bank: key = flips * n_cells + cell (see
// select_slice), and the slice of flip class x (bit 0) reads the other side
// with its columns reversed, of class y (bit 1) its rows reversed.  One
// thread per 8-element (16-byte) piece of a row: row r = (key * NL + lam,
// u, side), piece q; n_kl = slices of the stored bank x NL.
template <class TB>
__global__ void tr_bank_kernel(const TB* __restrict__ bank, unsigned short* __restrict__ bp,
                               int n_rows, int ks, int KP, int n_kl, bool f16) {
  const int per_row = KP / 8, total = n_rows * per_row;  // < 2^31 - 2^24 (checked on the host)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int r = i / per_row, q = i - r * per_row;
    const int side = r & 1, ru = r >> 1, u = ru % ks, klf = ru / ks;
    const int flips = klf / n_kl, kl = klf - flips * n_kl;
    const bool mx = flips & 1, my = flips & 2;
    const int sside = mx ? 1 - side : side, row = my ? u : ks - 1 - u;
    // element v of the flipped row: src[-v] (src[+v] for a column mirror)
    const TB* src = bank + (((size_t)kl * 2 + sside) * ks + row) * ks + (mx ? 0 : ks - 1);
    const int dir = mx ? 1 : -1;
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int v0 = 8 * q + 2 * k, v1 = v0 + 1;
      const float f0 = v0 < ks ? to_f32<TB>(src[dir * v0]) : 0.f;
      const float f1 = v1 < ks ? to_f32<TB>(src[dir * v1]) : 0.f;
      w[k] = (uint32_t)tc::to_op16(f0, f16) | ((uint32_t)tc::to_op16(f1, f16) << 16);
    }
    *reinterpret_cast<uint4*>(bp + (size_t)r * KP + 8 * q) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Bounded completion wait; a wait that gives up raises the launch's error
// flag at once, which makes every other wait of the launch give up too.
__device__ __forceinline__ bool wait_flag(uint64_t* bar, uint32_t parity, int* err,
                                          uint32_t limit) {
  if (tc::mbar_wait(bar, parity, limit, err)) return true;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// The render of one tile of 32 rows x 16 columns (4 blocks of 4 columns) of
// one channel.  For kernel row u and slice row n = (shift i, side, slot):
//   D[(g, cb), n] += sum_w Ipad[y0+g+u, x0+4cb+w] * Kf_(side,slot)[u][w-i]
// so D[(g, cb), (i, side, slot)] is the output of pixel (y0+g, x0+4cb+i).
// A (128 x K) is the image tile staged once with its 4 column blocks as
// consecutive 16-byte rows (the operand of row u is the same buffer moved by
// u image rows); B (64 x K) is built per kernel row from the flipped bank
// rows: its row (i, side, slot) is the kernel row shifted right by i.
template <bool F16>
__global__ void __launch_bounds__(TR_NT, 2) render_tc_kernel(const RenderParams P,
                                                             const unsigned short* __restrict__ bp,
                                                             int* __restrict__ err,
                                                             uint32_t wlim) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ int s_uniq[TR_MAXK], s_wcnt[TR_NT / 32], s_nuniq;
  __shared__ unsigned s_bits[TR_WIN / 32];
  __shared__ int s_wpre[TR_WIN / 32], s_kmin, s_over;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_full[TR_NB], s_empty[TR_NB], s_acc, s_fin;
  const int ks = P.ks, p = (ks - 1) >> 1, KP = tr_kp(ks), KK = tr_kk(ks), KB = KK / 8,
            R = TR_Y + ks - 1;
  const uint32_t LBO_A = tr_lbo_a(ks), BBUF = (uint32_t)tr_b_bytes(ks);
  unsigned char* Asm = smem;
  unsigned char* Bsm = smem + tr_a_bytes(ks);
  // candidate keys of the tile, in the B ring (free until the passes start)
  int* s_cand = reinterpret_cast<int*>(Bsm);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * TR_XW, y0 = blockIdx.y * TR_Y;
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
  // 1. threads 0..127: A row m = tid (tensor-memory lane m) = tile row m / 4,
  // column block m % 4, pixels i = 0..3.  Depths are loaded first and used
  // after the staging loads below have been issued.
  const bool pix = tid < TR_M;
  const int yy = y0 + (tid >> 2), xb = x0 + TR_J * (tid & 3);
  float dep[TR_J];
#pragma unroll
  for (int i = 0; i < TR_J; ++i)
    dep[i] = (pix && yy < H && xb + i < W) ? P.depth[((size_t)n * H + yy) * W + xb + i] : 1.f;

  // 2. stage the image tile: 16-byte row (image row r, block cb) of K block
  // kb holds Ipad[y0 + r][x0 + 4 cb + 8 kb + e], e = 0..7.  Every thread
  // first loads the 20 image values of each of its (row, K block) items
  // (packed in pairs), then stores the 4 rows of each.
  const unsigned short* img =
      reinterpret_cast<const unsigned short*>(P.aif) + ((size_t)n * P.C + c) * H * W;
  const int nitem = R * KB;  // <= TR_SI * TR_NT (checked on the host)
  uint32_t raw[TR_SI][10];
#pragma unroll
  for (int q = 0; q < TR_SI; ++q) {
    const int pr = tid + q * TR_NT;
    if (pr < nitem) {
      const int r = pr / KB, kb = pr - r * KB;
      const size_t rowoff = (size_t)min(max(y0 + r - p, 0), H - 1) * W;
      const int xs = x0 + 8 * kb - p;  // image column of element 0
      const unsigned short* src0 = img + rowoff + xs;
      if (xs >= 0 && xs + 20 <= W && (reinterpret_cast<uintptr_t>(src0) & 7) == 0) {
#pragma unroll
        for (int w = 0; w < 5; ++w) {
          const uint2 d = *reinterpret_cast<const uint2*>(src0 + 4 * w);
          raw[q][2 * w] = d.x;
          raw[q][2 * w + 1] = d.y;
        }
      } else {
#pragma unroll
        for (int w = 0; w < 10; ++w) {
          const uint32_t lo = img[rowoff + min(max(xs + 2 * w, 0), W - 1)];
          const uint32_t hi = img[rowoff + min(max(xs + 2 * w + 1, 0), W - 1)];
          raw[q][w] = lo | (hi << 16);
        }
      }
    }
  }
  int key[TR_J];
  float tt[TR_J];
  unsigned use = 0;  // bit 2i: slice key of pixel i used, bit 2i+1: key + 1
  int kmin_t = 0x7fffffff;
#pragma unroll
  for (int i = 0; i < TR_J; ++i) {
    key[i] = -1;
    tt[i] = 0.f;
    if (pix && yy < H && xb + i < W) {
      select_slice(P, yy, xb + i, dep[i], &key[i], &tt[i]);
      const bool u0 = !two || tt[i] < 1.f, u1 = two && tt[i] > 0.f;
      use |= (u0 ? 1u : 0u) << (2 * i);
      use |= (u1 ? 1u : 0u) << (2 * i + 1);
      kmin_t = min(kmin_t, u0 ? key[i] : key[i] + 1);
    }
  }
  if (pix && SD_CHECK(TR_J * 2 * tid + 2 * TR_J - 1, TR_MAXK)) {
#pragma unroll
    for (int i = 0; i < TR_J; ++i) {
      s_cand[TR_J * 2 * tid + 2 * i] = (use >> (2 * i)) & 1u ? key[i] : -1;
      s_cand[TR_J * 2 * tid + 2 * i + 1] = (use >> (2 * i + 1)) & 1u ? key[i] + 1 : -1;
    }
    if (use) atomicMin(&s_kmin, kmin_t);
  }
#pragma unroll
  for (int q = 0; q < TR_SI; ++q) {
    const int pr = tid + q * TR_NT;
    if (pr < nitem) {
      const int r = pr / KB, kb = pr - r * KB;
      unsigned char* dst = Asm + (size_t)kb * LBO_A + (size_t)r * TR_CB * 16;
#pragma unroll
      for (int cb = 0; cb < TR_CB; ++cb)
        *reinterpret_cast<uint4*>(dst + cb * 16) =
            make_uint4(raw[q][2 * cb], raw[q][2 * cb + 1], raw[q][2 * cb + 2], raw[q][2 * cb + 3]);
    }
  }
  if (warp == 0) tc::tmem_alloc(&s_tmem, TR_N);
  if (tid == 0) {
    for (int b = 0; b < TR_NB; ++b) {
      tc::mbar_init(&s_full[b], 32);
      tc::mbar_init(&s_empty[b], 1);
    }
    tc::mbar_init(&s_acc, 1);
    tc::mbar_init(&s_fin, 1);
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
  for (int q = tid; q < TR_MAXK; q += TR_NT) {
    const int kq = s_cand[q];
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
        if (SD_CHECK(pos, TR_MAXK)) s_uniq[pos] = kmin + 32 * w + bit;
        ++pos;
      }
    }
  } else {
    // first occurrences in candidate order; thread tid owns candidates
    // 4 tid .. 4 tid + 3
    constexpr int CPT = TR_MAXK / TR_NT;
    int cnt = 0;
    bool f[CPT];
#pragma unroll
    for (int e = 0; e < CPT; ++e) {
      const int q = CPT * tid + e, kq = s_cand[q];
      f[e] = kq >= 0;
      for (int m = 0; m < q && f[e]; ++m) f[e] = s_cand[m] != kq;
      cnt += f[e] ? 1 : 0;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_wcnt[warp] = incl;
    __syncthreads();
    int pos = incl - cnt;
    for (int w = 0; w < warp; ++w) pos += s_wcnt[w];
#pragma unroll
    for (int e = 0; e < CPT; ++e)
      if (f[e]) s_uniq[pos++] = s_cand[CPT * tid + e];
    if (tid == TR_NT - 1) s_nuniq = pos;
  }
  __syncthreads();  // s_cand is dead from here on (the B ring reuses it)
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
  int idx0[TR_J], idx1[TR_J];
  float w0[TR_J], w1[TR_J];
#pragma unroll
  for (int i = 0; i < TR_J; ++i) {
    idx0[i] = (use >> (2 * i)) & 1u ? slot_of(key[i]) : -1;
    idx1[i] = (use >> (2 * i + 1)) & 1u ? slot_of(key[i] + 1) : -1;
    w0[i] = two ? 1.f - tt[i] : 1.f;
    w1[i] = tt[i];
  }

  // 4. passes of up to 8 slices, one chunk per kernel row.  Producer warp
  // 4 + b builds the chunks of ring buffer b from the bank rows in global
  // memory (loaded one chunk ahead) and reports it full on its mbarrier;
  // thread 0 waits for a full buffer, issues its MMAs and lets the tensor
  // core report the buffer empty again.  At the end of a pass the tensor
  // core reports the accumulator, warps 0..3 fold it into their pixels and
  // meet at a named barrier before thread 0 starts the next pass.
  const int nch = ks, npass = (nuniq + TR_SL - 1) / TR_SL, total = npass * nch;
  const uint32_t idesc = F16 ? tc::idesc_f16_f32(TR_M, TR_N) : tc::idesc_bf16_f32(TR_M, TR_N);
  const uint32_t a_base = tc::smem_u32(Asm), b_base = tc::smem_u32(Bsm);
  const uint64_t a_desc0 = tc::smem_desc(a_base, LBO_A, 128);
  const uint64_t b_desc0 = tc::smem_desc(b_base, TR_N * 16, 128);
  float outL[TR_J], outR[TR_J];
#pragma unroll
  for (int i = 0; i < TR_J; ++i) outL[i] = outR[i] = 0.f;
  if (warp >= TR_CB) {
    // producer: task e = lane + 32 q of a chunk is (K block kb = e / 16,
    // row ss = e % 16 = side * 8 + slot); it writes the rows (i, ss) of K
    // block kb for the 4 shifts i from the bank words kb - 1 and kb.  A lane
    // loads word kb of its tasks (one chunk ahead) and takes word kb - 1
    // from the lane of task e - 16.
    const int b = warp - TR_CB;
    const uint32_t bdst = b_base + (uint32_t)b * BBUF;
    const int ntask = TR_SS * KB, qwords = KP / 8;
    uint4 cur[TR_TPL], nxt[TR_TPL];
    auto load = [&](uint4 (&dst)[TR_TPL], int cg) {
      const int pass = cg / nch, u = cg - pass * nch;
#pragma unroll
      for (int q = 0; q < TR_TPL; ++q) {
        const int e = lane + 32 * q, kb = e >> 4, ss = e & 15;
        const int ui = pass * TR_SL + (ss & 7);
        dst[q] = make_uint4(0u, 0u, 0u, 0u);
        if (e < ntask && ui < nuniq && kb < qwords)
          dst[q] = __ldg(reinterpret_cast<const uint4*>(
              bp + (((long long)s_uniq[ui] * P.NL + lam) * ks + u) * 2 * KP + (ss >> 3) * KP +
              8 * kb));
      }
    };
    auto shfl4 = [&](const uint4& v) {
      uint4 r;
      r.x = __shfl_xor_sync(0xffffffffu, v.x, 16);
      r.y = __shfl_xor_sync(0xffffffffu, v.y, 16);
      r.z = __shfl_xor_sync(0xffffffffu, v.z, 16);
      r.w = __shfl_xor_sync(0xffffffffu, v.w, 16);
      return r;
    };
    if (b < total) load(cur, b);
    for (int cg = b; cg < total; cg += TR_NB) {
      if (cg + TR_NB < total) load(nxt, cg + TR_NB);
      if (cg >= TR_NB)  // the MMAs of chunk cg - TR_NB read this buffer
        wait_flag(&s_empty[b], (uint32_t)(cg / TR_NB - 1) & 1u, err, wlim);
      const int ui_base = (cg / nch) * TR_SL;
      uint4 other = make_uint4(0u, 0u, 0u, 0u);  // word kb of task e - 16 + 32 (q - 1)
#pragma unroll
      for (int q = 0; q < TR_TPL; ++q) {
        const uint4 same = shfl4(cur[q]);  // word kb of task e + 16 or e - 16 (same q)
        const uint4 prev = lane >= 16 ? same : other;
        other = same;
        const int e = lane + 32 * q, kb = e >> 4, ss = e & 15;
        if (e < ntask && ui_base + (ss & 7) < nuniq) {
          // elements 8 kb - i .. 8 kb - i + 7 of the row: the 16 elements of
          // words kb - 1 and kb from position 8 - i on
          const uint32_t c8[8] = {prev.x, prev.y, prev.z, prev.w,
                                  cur[q].x, cur[q].y, cur[q].z, cur[q].w};
          const uint32_t d = bdst + (uint32_t)kb * (TR_N * 16) + (uint32_t)ss * 16;
#pragma unroll
          for (int i = 0; i < TR_J; ++i) {
            uint32_t g[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              if (i & 1)
                g[k] = __funnelshift_r(c8[(7 - i) / 2 + k], c8[(9 - i) / 2 + k], 16);
              else
                g[k] = c8[(8 - i) / 2 + k];
            }
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(d + i * TR_SS * 16),
                         "r"(g[0]), "r"(g[1]), "r"(g[2]), "r"(g[3])
                         : "memory");
          }
        }
      }
      tc::fence_async_smem();
      tc::mbar_arrive(&s_full[b]);
#pragma unroll
      for (int q = 0; q < TR_TPL; ++q) cur[q] = nxt[q];
    }
  } else {
    // thread 0 stops issuing products at the first wait that gives up (the
    // launch's error flag is then set and its output invalid)
    bool issuing = true;
    for (int pass = 0; pass < npass; ++pass) {
      if (tid == 0) {
        for (int ch = 0; ch < nch && issuing; ++ch) {
          const int cg = pass * nch + ch, b = cg % TR_NB;
          issuing = wait_flag(&s_full[b], (uint32_t)(cg / TR_NB) & 1u, err, wlim);
          if (!issuing) break;
          tc::fence_after_sync();
          // the start-address field is the low 14 bits (address >> 4)
          uint64_t ad = a_desc0 + (uint64_t)(ch * TR_CB);  // rows of 64 B
          uint64_t bd = b_desc0 + (uint64_t)((uint32_t)b * BBUF >> 4);
          for (int kq = 0; kq < KK / 16; ++kq) {
            tc::mma_bf16(tmem, ad, bd, idesc, !(ch == 0 && kq == 0));
            ad += (uint64_t)(2u * LBO_A >> 4);
            bd += (uint64_t)(2u * TR_N * 16 >> 4);
          }
          tc::commit(&s_empty[b]);
        }
        if (issuing) tc::commit(&s_acc);
      }
      __syncwarp();
      // the pass's accumulator; a warp reads tensor memory only when every
      // lane saw it complete (the loads are warp-collective)
      const bool got =
          __all_sync(0xffffffffu, wait_flag(&s_acc, (uint32_t)pass & 1u, err, wlim));
      tc::fence_after_sync();
#pragma unroll
      for (int i = 0; i < TR_J && got; ++i) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(i * TR_SS), v);
#pragma unroll
        for (int sl = 0; sl < TR_SL; ++sl) {
          const int ui = pass * TR_SL + sl;
          if (ui == idx0[i]) {
            outL[i] = fmaf(w0[i], v[sl], outL[i]);
            outR[i] = fmaf(w0[i], v[TR_SL + sl], outR[i]);
          }
          if (ui == idx1[i]) {
            outL[i] = fmaf(w1[i], v[sl], outL[i]);
            outR[i] = fmaf(w1[i], v[TR_SL + sl], outR[i]);
          }
        }
      }
      tc::fence_before_sync();
      named_sync(1, TR_M);
    }
    unsigned short* out = reinterpret_cast<unsigned short*>(P.out);
#pragma unroll
    for (int i = 0; i < TR_J; ++i)
      if (pix && yy < H && xb + i < W) {
        out[(((size_t)n * 2 * P.C + c) * H + yy) * W + xb + i] = tc::to_op16(outL[i], F16);
        out[(((size_t)n * 2 * P.C + P.C + c) * H + yy) * W + xb + i] =
            tc::to_op16(outR[i], F16);
      }
    // every product this CTA issued has completed before its tensor memory
    // is freed, also when a wait gave up (a commit tracks all of them; the
    // drain is bounded but not cut short by the error flag)
    if (tid == 0) {
      tc::commit(&s_fin);
      if (!tc::mbar_wait(&s_fin, 0, TR_DRAIN)) atomicExch(err, 1);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, TR_N);
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
                                     int image_dtype, void* out, void* workspace,
                                     size_t workspace_bytes, void* stream) {
  SD_API_RANGE("sd_dp_render_tc");
  using namespace sd;
  if (!aif || !depth_m || !bank || !out) return SD_ERR_ARG;
  if (N < 0 || C < 1 || H < 0 || W < 0) return SD_ERR_ARG;
  RenderParams P;
  std::memset(&P, 0, sizeof P);
  sd_status st = check_layout(layout, P);
  if (st != SD_OK) return st;
  if (image_dtype != SD_BF16 && image_dtype != SD_F16) return SD_ERR_UNSUPPORTED;
  const bool f16 = image_dtype == SD_F16;
  // the bank in the image's type, or FP32 (rounded to it by the re-layout)
  if (layout->dtype != image_dtype && layout->dtype != SD_F32) return SD_ERR_UNSUPPORTED;
  if (P.ks > 65 || tr_smem(P.ks) > 227 * 1024 ||
      (TR_Y + P.ks - 1) * (tr_kk(P.ks) / 8) > TR_SI * TR_NT || TR_SS * (tr_kk(P.ks) / 8) > 32 * TR_TPL)
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
  unsigned short* bp = reinterpret_cast<unsigned short*>(reinterpret_cast<char*>(workspace) + 256);
  SD_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  const long long n_rows = (long long)tr_slices(P) * P.NL * P.ks * 2;
  const int n_kl = P.FC * P.Z * P.NL;  // slices x wavelengths of the stored bank
  const int kp = tr_kp(P.ks);
  if (n_rows * (kp / 8) > 0x7f000000ll) return SD_ERR_UNSUPPORTED;
  const int pieces = (int)(n_rows * (kp / 8));
  const int nblk = std::min((pieces + 255) / 256, 152 * 16);
  if (layout->dtype == SD_BF16)
    tr_bank_kernel<__nv_bfloat16><<<nblk, 256, 0, s>>>(
        reinterpret_cast<const __nv_bfloat16*>(bank), bp, (int)n_rows, P.ks, kp, n_kl, false);
  else if (layout->dtype == SD_F16)
    tr_bank_kernel<__half><<<nblk, 256, 0, s>>>(reinterpret_cast<const __half*>(bank), bp,
                                                (int)n_rows, P.ks, kp, n_kl, true);
  else
    tr_bank_kernel<float><<<nblk, 256, 0, s>>>(reinterpret_cast<const float*>(bank), bp,
                                               (int)n_rows, P.ks, kp, n_kl, f16);
  st = launch_status();
  if (st != SD_OK) return st;
  const size_t smem = tr_smem(P.ks);
  auto k = f16 ? render_tc_kernel<true> : render_tc_kernel<false>;
  SD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((W + TR_XW - 1) / TR_XW, (H + TR_Y - 1) / TR_Y, N * C);
  k<<<grid, TR_NT, smem, s>>>(P, bp, err, wait_limit(TR_WAIT));
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

SD_CHECK_TU(render_tc)
