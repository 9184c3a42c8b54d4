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
// Kernels (every sum in a fixed order: both gradients are deterministic):
//   select_table_kernel     per pixel: its slice selection (key, t), once;
//   slice_bitmap_kernel     per (image, tile): which bank slices the tile uses
//                           (a bitmap in the caller's workspace);
//   render_bwd_img_kernel   per (strip of 64 source columns, 8 output rows,
//                           channel): warps scatter source blocks, slice by
//                           slice, into private row buffers added in warp
//                           order; strips whose footprints overlap run in
//                           separate launches (section 2);
//   slice_count_kernel,     the slices ordered by how many tiles use them
//   slice_order_kernel      (the heaviest first);
//   render_bwd_bank_kernel  per (slice, wavelength), in that order: visits, in
//                           a fixed order, the tiles whose bitmap holds the
//                           slice; threads own 8-tap strips of the kernel and
//                           accumulate over the tile's segments in a fixed
//                           order, then write the slice's gradient;
//   bank_grad_tc_kernel     the bank gradient on the tensor cores (section 4).

#define SD_TU 3  // translation unit id of this file's SD_CHECK sites
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
    selected(P, n, yy, xx, &key, &t);
    if (!two || t < 1.f) atomicOr(&sb[key >> 5], 1u << (key & 31));
    if (two && t > 0.f) atomicOr(&sb[(key + 1) >> 5], 1u << ((key + 1) & 31));
  }
  __syncthreads();
  size_t tile = ((size_t)n * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  for (int i = tid; i < words; i += NT_BM) bm[tile * words + i] = sb[i];
}

// ---------------------------------------------------------------------------
// 2. image gradient, deterministic.  A thread block owns a strip of IG_SW
// source columns of one channel and one 8-row block of output rows (image
// rows 8i .. 8i+7; the first and last blocks also take the padded rows that
// the replicate padding folds onto image rows 0 and H-1).  The 8-row source
// blocks within reach are dealt to its warps in turn; a warp stages a source
// block's selection and output gradients, finds the slices the block uses
// (ascending), and for each slice lets each lane take one source column that
// uses it: for every kernel
// column v the lane's 8 weighted gradients (both sides) meet the 15 kernel
// rows that connect its 8 source rows to the 8 output rows,
//   dIpad[T0 + j][x + v] += sum_a w_k G_s(8 sb + a, x) Kf_{k,s}[d + j - a][v],
// d = T0 + p - 8 sb, and the lane adds its 8 sums to its column of a
// warp-private row buffer (one plain read-modify-write per row: the lanes of
// a pass own distinct columns, and the warp's steps run in program order).
// The buffers cover the strip's footprint (IG_SW + ks - 1 columns); at the
// end they are added in warp order and the sum is added to the image once.  Strips whose footprints overlap run
// in different launches (phases), so no two warps of a launch write the
// same image element and every element receives its phase contributions in
// a fixed order: bitwise reproducible, no atomics.
//   Taps come from a per-call re-layout of the bank: per (slice key,
// wavelength) and flipped-kernel column v, the column's rows (both sides
// interleaved, zero-padded above and below) as 16-byte aligned runs, so the
// 15 rows of a band are 8 broadcast 16-byte loads; a table of each row's
// non-zero column range bounds the kernel columns a band visits.
// ---------------------------------------------------------------------------
constexpr int IG_SW = 64;   // source columns per warp (two per lane)
constexpr int IG_NW = 4;    // warps per block (one item, private buffers)
constexpr unsigned short IG_EMPTY = 0x00ffu;  // row extent of an all-zero row

struct ImgLayout {
  int padu;    // zero rows above kernel row 0 in a re-laid column
  int rcol;    // rows per re-laid column (even)
  int nphase;  // launches of non-overlapping strips
  size_t kcol_bytes, ext_bytes, total;
};

// Bytes of the per-pixel selection table (first in every backward
// workspace: both gradient passes and the bitmap read it).
inline size_t sel_table_bytes(const RenderParams& P) {
  return ((size_t)P.N * P.H * P.W * 8 + 255) & ~(size_t)255;
}

inline ImgLayout img_layout(const RenderParams& P) {
  ImgLayout L;
  const int ks = P.ks, p = (ks - 1) / 2;
  // bands start at row d - 7 with d = p (mod 8) and d in [-7, ks + 6]: the
  // padding keeps every band inside its column and 16-byte aligned
  L.padu = (p & 1) ? 14 : 15;
  L.rcol = (ks + 15 + L.padu + 1) & ~1;
  L.nphase = 1 + (2 * p + IG_SW - 1) / IG_SW;
  const size_t kl = (size_t)n_keys(P) * P.NL;
  L.kcol_bytes = (kl * ks * L.rcol * 8 + 255) & ~(size_t)255;
  L.ext_bytes = (kl * ks * 2 + 255) & ~(size_t)255;
  L.total = L.kcol_bytes + L.ext_bytes;
  return L;
}

// Per-pixel selection (key, t) of every pixel, once per call.
__global__ void select_table_kernel(const RenderParams P, int2* __restrict__ sel) {
  const size_t npx = (size_t)P.N * P.H * P.W;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npx;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % P.W);
    const size_t r = i / P.W;
    const int y = (int)(r % P.H);
    int key;
    float t;
    select_slice(P, y, x, P.depth[i], &key, &t);
    sel[i] = make_int2(key, __float_as_int(t));
  }
}

// Re-layout of one (slice key, wavelength) per block: the flipped kernel
// Kf_s[u][v] (quadrant banks: the key's flip class, see select_slice) as
// kcol[kl][v][padu + u][s], zero outside 0 <= u < ks, and each row's
// non-zero column range ext[kl][u] = vlo | vhi << 8 (IG_EMPTY if none).
template <class TB>
__global__ void __launch_bounds__(256) kernel_columns_kernel(const RenderParams P,
                                                             ImgLayout IL,
                                                             float* __restrict__ kcol,
                                                             unsigned short* __restrict__ ext) {
  extern __shared__ __align__(16) float kf[];  // [2][ks][ks]
  const int ks = P.ks, ks2 = ks * ks, kl = blockIdx.x;
  const int n_kl = P.FC * P.Z * P.NL;  // slices x wavelengths of the stored bank
  const int flips = kl / n_kl, kls = kl - flips * n_kl;
  const bool mx = flips & 1, my = flips & 2;
  const TB* src = reinterpret_cast<const TB*>(P.bank) + (size_t)kls * 2 * ks2;
  for (int i = threadIdx.x; i < 2 * ks2; i += blockDim.x) {
    const int s = i / ks2, r = i - s * ks2, row = r / ks, col = r - row * ks;
    // stored (side s, row, col) is flipped element (u, v) of side s' below
    const int u = my ? row : ks - 1 - row, v = mx ? col : ks - 1 - col;
    const int sf = mx ? 1 - s : s;
    kf[(sf * ks + u) * ks + v] = to_f32<TB>(src[i]);
  }
  __syncthreads();
  float* dst = kcol + (size_t)kl * ks * IL.rcol * 2;
  for (int i = threadIdx.x; i < ks * IL.rcol * 2; i += blockDim.x) {
    const int v = i / (IL.rcol * 2), q = i - v * IL.rcol * 2, rho = q >> 1, s = q & 1;
    const int u = rho - IL.padu;
    if (SD_CHECK((size_t)kl * ks * IL.rcol * 2 + i, IL.kcol_bytes / 4))
      dst[i] = (u >= 0 && u < ks) ? kf[(s * ks + u) * ks + v] : 0.f;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int u = warp; u < ks; u += blockDim.x / 32) {
    unsigned lo = 255u, hi = 0u;
    for (int v = lane; v < ks; v += 32)
      if (kf[u * ks + v] != 0.f || kf[(ks + u) * ks + v] != 0.f) {
        lo = min(lo, (unsigned)v);
        hi = max(hi, (unsigned)v);
      }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) ext[(size_t)kl * ks + u] = (unsigned short)(lo > hi ? IG_EMPTY : lo | (hi << 8));
  }
}

// position of the idx-th (0-based) set bit of m (idx < popc(m))
__device__ __forceinline__ int nth_set_bit(unsigned m, int idx) {
  int pos = 0;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const int c = __popc(m & ((1u << s) - 1u));
    if (idx >= c) {
      idx -= c;
      m >>= s;
      pos += s;
    }
  }
  return pos;
}

// A half pass: up to 16 candidate columns of one slice (the columns of the
// staged source block whose pixels use the slice: bit c of m0 is column c,
// bit c of m1 column 32 + c), candidates q0 .. q0 + 15 of them.  Warp-uniform.
struct IgUnit {
  int k;              // slice key
  int vlo, vhi;       // kernel columns holding a non-zero tap in the band
  unsigned m0, m1;
  int n0, ncand, q0;  // n0 = popc(m0); ncand = candidates of the slice
  const float* kb0;   // re-laid taps of kernel column vlo, band start
};

// One pass: lanes 0-15 take unit U0's candidates into row buffer buf0,
// lanes 16-31 unit U1's (if valid) into buf1.  Each lane holds 8 source
// rows of its column, weighted by the slice's interpolation weight, and
// for every kernel column v of the union of the two units' ranges (taps
// outside a unit's range are zero) adds the 8 output rows of the band to
// its buffer column.  Within a half the columns are distinct, and the two
// halves write separate buffers, so no two lanes touch one word.
template <int BWMAX>
__device__ __forceinline__ void ig_pass(const float4 (*src)[IG_SW], float* buf0, float* buf1,
                                        const IgUnit& U0, const IgUnit& U1, bool u1_valid,
                                        bool two, bool plain, int jr0, int fold_lo, int fold_hi,
                                        size_t col_stride) {
  const int lane = threadIdx.x & 31, h = lane >> 4;
  const bool mine_valid = h == 0 || u1_valid;
  // this lane's unit (selected field by field: the values are warp-uniform
  // per half)
  const int k = h ? U1.k : U0.k;
  const unsigned m0 = h ? U1.m0 : U0.m0, m1 = h ? U1.m1 : U0.m1;
  const int n0 = h ? U1.n0 : U0.n0, ncand = h ? U1.ncand : U0.ncand;
  // an idle half (no second unit) keeps the first unit's range and taps so
  // that its loads stay inside the re-laid bank
  const bool hu = h && u1_valid;
  const int vlo_u = hu ? U1.vlo : U0.vlo;
  const float* kb_u = hu ? U1.kb0 : U0.kb0;
  const int idx = (h ? U1.q0 : U0.q0) + (lane & 15);
  const bool act = mine_valid && idx < ncand;
  const int col = !act ? 0 : (idx < n0 ? nth_set_bit(m0, idx) : 32 + nth_set_bit(m1, idx - n0));
  const int vlo = u1_valid ? min(U0.vlo, U1.vlo) : U0.vlo;
  const int vhi = u1_valid ? max(U0.vhi, U1.vhi) : U0.vhi;
  // (L, R) pairs: the weighted gradients, the re-laid taps (interleaved by
  // side) and the sums go through the packed two-lane FMA, whose components
  // round like fmaf (the same sums, half the FMA instructions)
  float2 G2[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const float4 e = src[a][col];
    const int k0 = __float_as_int(e.w);
    const float w = !act || k0 < 0 ? 0.f
                    : (k0 == k ? (two ? 1.f - e.z : 1.f) : ((two && k0 + 1 == k) ? e.z : 0.f));
    G2[a] = make_float2(w * e.x, w * e.y);
  }
  // the lane reads its own unit's taps from column vlo (of the union) on;
  // columns before its own range are zero, so start the pointer there too
  const size_t cs4 = col_stride / 4;
  const float4* kb = reinterpret_cast<const float4*>(kb_u) - (ptrdiff_t)(vlo_u - vlo) * cs4;
  float* bcol = (h ? buf1 : buf0) + col;
  // taps of column v: rows d - 7 .. d + 8, (L, R) interleaved; the next
  // column's are loaded while this one is used
  float4 tn[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) tn[q] = __ldg(kb + q);
  for (int v = vlo; v <= vhi; ++v) {
    float2 T2[16];  // band row r: (L, R)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      T2[2 * q] = make_float2(tn[q].x, tn[q].y);
      T2[2 * q + 1] = make_float2(tn[q].z, tn[q].w);
    }
    kb += cs4;
    if (v < vhi) {
#pragma unroll
      for (int q = 0; q < 8; ++q) tn[q] = __ldg(kb + q);
    }
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < 8; ++a) s2 = __ffma2_rn(G2[a], T2[j - a + 7], s2);
      acc[j] = s2.x + s2.y;
    }
    if (act && SD_CHECK(col + v, BWMAX)) {
      if (plain) {  // distinct rows: loads, adds and stores batch
        float old8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) old8[j] = bcol[j * BWMAX + v];
#pragma unroll
        for (int j = 0; j < 8; ++j) bcol[j * BWMAX + v] = old8[j] + acc[j];
      } else {  // folded rows may repeat: in order, one at a time
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int tr = min(max(jr0 + j, fold_lo), fold_hi);
          if (SD_CHECK(tr, 8)) bcol[tr * BWMAX + v] += acc[j];
        }
      }
    }
    __syncwarp();
  }
}

template <int BWMAX>
__global__ void __launch_bounds__(IG_NW * 32, 3) render_bwd_img_kernel(
    const RenderParams P, ImgLayout IL, const float* __restrict__ gout,
    const int2* __restrict__ sel, const float* __restrict__ kcol,
    const unsigned short* __restrict__ ext, int phase, int nr_phase, int nrb,
    float* __restrict__ gaif) {
  // per warp: the staged source block (gL, gR, t, key) and a row buffer per
  // half-warp
  extern __shared__ __align__(16) unsigned char smem[];
  float4 (*s_src)[8][IG_SW] = reinterpret_cast<float4 (*)[8][IG_SW]>(smem);
  // buffer b = 2 * warp + half at s_buf + b * IG_BUFS: 16 floats of padding
  // put a column's word in the two halves' buffers in different banks
  constexpr int IG_BUFS = 8 * BWMAX + 16;
  float* s_buf = reinterpret_cast<float*>(smem + (size_t)IG_NW * 8 * IG_SW * 16);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // one item (strip of source columns, 8 output rows) per block
  const long long item = blockIdx.x;
  const int rr = (int)(item % nr_phase);
  const long long rest = item / nr_phase;
  const int rb = (int)(rest % nrb);
  const int nc = (int)(rest / nrb);
  const int n = nc / P.C, c = nc - n * P.C;
  const int lam = (P.NL == P.C) ? c : 0;
  const int H = P.H, W = P.W, ks = P.ks, p = (ks - 1) >> 1;
  const int x0 = (phase + IL.nphase * rr) * IG_SW;
  const int BW = IG_SW + ks - 1;
  const bool two = P.Z > 1;
  float* buf0 = s_buf + (size_t)(2 * warp) * IG_BUFS;
  float* buf1 = buf0 + IG_BUFS;
  float4 (*src)[IG_SW] = s_src[warp];
  for (int i = lane; i < 2 * IG_BUFS; i += 32) buf0[i] = 0.f;  // both halves

  const float* goL = gout + (((size_t)n * 2 * P.C + c) * H) * W;
  const float* goR = gout + (((size_t)n * 2 * P.C + P.C + c) * H) * W;
  const int2* selp = sel + (size_t)n * H * W;
  const int nsb = (H + 7) >> 3;
  const int r0 = 8 * rb;
  // virtual output row groups T0 = r0 + 8 g: rows above the image fold onto
  // row 0 (first block), rows below onto row H - 1 (last block)
  const int g_lo = rb == 0 ? -((p + 7) >> 3) : 0;
  const int g_hi = r0 + 8 >= H ? (H - 1 + p - r0) >> 3 : 0;
  const size_t col_stride = (size_t)IL.rcol * 2;  // floats per re-laid column
  const int fold_lo = -r0, fold_hi = H - 1 - r0;  // buffer rows of clamped rows

  // the (group, source block) pairs of the item: the first pairs are dealt
  // to the warps in turn, the last npairs mod IG_NW are shared by all warps,
  // each taking every IG_NW-th of the pair's slices (a fixed assignment, so
  // the buffers' sums do not vary; without the sharing an interior item's 9
  // pairs left one warp with 3 while the others waited at the barrier)
  int npairs = 0;
  for (int g = g_lo; g <= g_hi; ++g) {
    const int T0 = r0 + 8 * g;
    npairs += max(0, min(nsb - 1, (T0 + 7 + p) >> 3) - max(0, (T0 - p) >> 3) + 1);
  }
  const int dealt = npairs - npairs % IG_NW;
  int pair = 0;
  for (int g = g_lo; g <= g_hi; ++g) {
    const int T0 = r0 + 8 * g;
    const bool plain = T0 == r0 && r0 + 8 <= H;  // no row folds
    // source blocks within reach: rows T0 - p .. T0 + 7 + p
    const int sb_lo = max(0, (T0 - p) >> 3);  // arithmetic shift: floor division
    const int sb_hi = min(nsb - 1, (T0 + 7 + p) >> 3);
    for (int sb = sb_lo; sb <= sb_hi; ++sb, ++pair) {
      const bool shared_pair = pair >= dealt;
      if (!shared_pair && pair % IG_NW != warp) continue;
      const int d = T0 + p - 8 * sb;  // kernel row of (j, a) = d + j - a
      // stage the source block: lane owns columns lane and lane + 32
      __syncwarp();
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int y = 8 * sb + a;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int col = lane + 32 * h, x = x0 + col;
          float4 e = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
          if (y < H && x < W) {
            const size_t o = (size_t)y * W + x;
            const int2 sv = selp[o];
            e = make_float4(goL[o], goR[o], __int_as_float(sv.y), __int_as_float(sv.x));
          }
          src[a][col] = e;
        }
      }
      __syncwarp();
      // the block's slices in ascending order; a pixel (key k0, weight t)
      // uses k0 unless t == 1 and k0 + 1 when t > 0 (one slice: k0 only)
      int last = -1, ordinal = 0;
      bool pending = false;  // a half pass waiting for its partner
      IgUnit held{};
      while (true) {
        int m = 0x7fffffff;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float4 e = src[q >> 1][lane + 32 * (q & 1)];
          const int k0 = __float_as_int(e.w);
          if (k0 >= 0) {
            if ((!two || e.z < 1.f) && k0 > last) m = min(m, k0);
            if (two && e.z > 0.f && k0 + 1 > last) m = min(m, k0 + 1);
          }
        }
        const int k = __reduce_min_sync(0xffffffffu, m);
        if (k == 0x7fffffff) break;
        last = k;
        if (shared_pair && ordinal++ % IG_NW != warp) continue;
        const int kl = k * P.NL + lam;
        // kernel columns holding a non-zero tap in rows d - 7 .. d + 7
        unsigned lo = 255u, hi = 0u;
        if (lane < 15) {
          const int u = d - 7 + lane;
          if (u >= 0 && u < ks) {
            const unsigned e = ext[(size_t)kl * ks + u];
            lo = e & 0xffu;
            hi = e >> 8;
          }
        }
        const int vlo = (int)__reduce_min_sync(0xffffffffu, lo);
        const int vhi = (int)__reduce_max_sync(0xffffffffu, hi);
        if (vlo > vhi) continue;
        // the lane's columns that use slice k
        bool f0 = false, f1 = false;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float4 e = src[q >> 1][lane + 32 * (q & 1)];
          const int k0 = __float_as_int(e.w);
          const bool use = k0 >= 0 && (((!two || e.z < 1.f) && k0 == k) ||
                                       (two && e.z > 0.f && k0 + 1 == k));
          if (q & 1) f1 = f1 || use; else f0 = f0 || use;
        }
        const unsigned m0 = __ballot_sync(0xffffffffu, f0);
        const unsigned m1 = __ballot_sync(0xffffffffu, f1);
        const int n0 = __popc(m0), ncand = n0 + __popc(m1);
        // the slice's candidates in half passes of 16, paired in order (the
        // band of the slice's last kernel column stays inside the re-laid bank)
        if (!SD_CHECK(((size_t)kl * ks + ks - 1) * col_stride + 2 * (d - 7 + IL.padu) + 31,
                      IL.kcol_bytes / 4))
          continue;
        const IgUnit U{k, vlo, vhi, m0, m1, n0, ncand, 0,
                       kcol + ((size_t)kl * ks + vlo) * col_stride + 2 * (d - 7 + IL.padu)};
        for (int q0 = 0; q0 < ncand; q0 += 16) {
          IgUnit u = U;
          u.q0 = q0;
          if (!pending) {
            held = u;
            pending = true;
          } else {
            ig_pass<BWMAX>(src, buf0, buf1, held, u, true, two, plain, T0 - r0, fold_lo,
                           fold_hi, col_stride);
            pending = false;
          }
        }
      }
      if (pending)
        ig_pass<BWMAX>(src, buf0, buf1, held, held, false, two, plain, T0 - r0, fold_lo,
                       fold_hi, col_stride);
    }
  }
  __syncthreads();
  // the buffers added in (warp, half) order into the first
  float* b0 = s_buf;
  for (int i = threadIdx.x; i < 8 * BWMAX; i += IG_NW * 32) {
    float s = b0[i];
#pragma unroll
    for (int w = 1; w < 2 * IG_NW; ++w) s += s_buf[(size_t)w * IG_BUFS + i];
    b0[i] = s;
  }
  float (*fb)[BWMAX] = reinterpret_cast<float (*)[BWMAX]>(b0);  // [8][BWMAX]
  __syncthreads();
  // columns outside the image fold onto its first / last column (fixed order)
  const int cl = p - x0;            // buffer column of image column 0
  const int cr = W - 1 - x0 + p;    // buffer column of image column W - 1
  if (threadIdx.x < 8) {
    const int j = threadIdx.x;
    if (cl > 0) {
      float s = 0.f;
      for (int cc = 0; cc <= cl; ++cc) s += fb[j][cc];
      fb[j][cl] = s;
    }
    if (cr < BW - 1) {
      float s = fb[j][cr];
      for (int cc = cr + 1; cc < BW; ++cc) s += fb[j][cc];
      fb[j][cr] = s;
    }
  }
  __syncthreads();
  float* ga = gaif + ((size_t)n * P.C + c) * H * W;
  const int nrow = min(8, H - r0);
  const int c_lo = max(0, cl), c_hi = min(BW - 1, cr);
  const int ncol = c_hi - c_lo + 1;
  for (int i = threadIdx.x; i < nrow * ncol; i += IG_NW * 32) {
    const int j = i / ncol, cc = c_lo + (i - j * ncol);
    const long long o = (long long)(r0 + j) * W + (x0 - p + cc);
    if (SD_CHECK(o, (long long)H * W) && SD_CHECK(cc, BWMAX)) ga[o] += fb[j][cc];
  }
}

// ---------------------------------------------------------------------------
// 3. bank gradient, one block per (slice key, wavelength)
// ---------------------------------------------------------------------------
// Work plan of a bank-gradient launch (built on the device by
// slice_count_kernel and slice_order_kernel, in the caller's workspace).
struct BankPlan {
  const int* order;  // item of each block rank: key * 2 + chunk; -1 past the last
  const int* slot;   // split slot of a key, -1 for a slice that is one item
  int* tick;         // per (split slot, wavelength): chunks finished
  float* pbuf;       // per (split slot, chunk, wavelength): a 2 ks^2 slab
  int nkeys;
  int smax;          // split slots
  __device__ float* slab(int sl, int chunk, int lam, int NL, int ks2) const {
    return pbuf + (((size_t)sl * 2 + chunk) * NL + lam) * 2 * (size_t)ks2;
  }
};

// The tiles t0 .. t0 + NT - 1 (of ntiles) of the block's chunk (all tiles,
// or those with index = chunk mod 2) whose bitmap holds the slice, as
// offsets from t0 in ascending order: one tile per thread, compacted with
// warp ballots, so that the bitmap loads of NT tiles are in flight together
// (a scan of one tile after the other waits for each load in turn).  Every
// thread of the block calls it; returns the count.
template <int NT>
__device__ int slice_tiles(const unsigned* __restrict__ bm, int words, int kw, unsigned kbit,
                           size_t t0, size_t ntiles, int nch, int chunk, int* s_list,
                           int* s_wc) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t t = t0 + tid;
  const bool use = t < ntiles && (nch == 1 || (int)(t & 1) == chunk) &&
                   (bm[t * words + kw] & kbit) != 0u;
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

// Tiles per key (how many tiles' bitmaps hold it): block (word, chunk of
// 1024 tiles), counts by warp ballots, integer atomics into cnt (zeroed by
// the caller; the sums do not depend on the order).
__global__ void __launch_bounds__(256) slice_count_kernel(const unsigned* __restrict__ bm,
                                                          int words, size_t ntiles, int nkeys,
                                                          int* __restrict__ cnt) {
  __shared__ int s_c[8][32];
  const int w = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t t0 = (size_t)blockIdx.y * 1024 + threadIdx.x;
  int mine = 0;  // lane b: tiles of this warp holding bit b
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const size_t t = t0 + 256 * i;
    const unsigned x = t < ntiles ? bm[t * words + w] : 0u;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      const int c = __popc(__ballot_sync(0xffffffffu, (x >> b) & 1u));
      mine += lane == b ? c : 0;
    }
  }
  s_c[warp][lane] = mine;
  __syncthreads();
  if (warp == 0) {
    int sum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) sum += s_c[q][lane];
    const int key = w * 32 + lane;
    if (sum && key < nkeys) atomicAdd(cnt + key, sum);
  }
}

// Work plan of the bank-gradient blocks (one block per item and wavelength).
// A slice whose tile count exceeds half a block's fair share (NL x all
// counts / the resident blocks) is split into two items, chunk c taking its
// tiles with index = c (mod 2), as long as split slots remain (in key
// order); every other slice is one item.  Items are ordered by descending tile
// count per item (64 buckets of the count; ascending item id within a
// bucket) so that the largest start first and none is left to run alone at
// the end (longest-processing-time order).  order[i] = key * 2 + chunk, -1
// past the last item; slot[key] = the split slot or -1.  One block of 1024
// threads; everything it decides follows from the counts (deterministic).
__global__ void __launch_bounds__(1024) slice_order_kernel(const int* __restrict__ cnt,
                                                           int nkeys, int NL, int resident,
                                                           int smax, int* __restrict__ slot,
                                                           int* __restrict__ split_key,
                                                           int* __restrict__ order) {
  constexpr int NB = 64;
  __shared__ int s_hist[NB], s_base[NB], s_tot[NB], s_wc[32][NB], s_max[32], s_n[32];
  __shared__ long long s_sum[32];
  __shared__ int s_run;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int m = 0;
  long long sum = 0;
  for (int k = tid; k < nkeys; k += 1024) {
    m = max(m, cnt[k]);
    sum += cnt[k];
  }
  m = __reduce_max_sync(0xffffffffu, m);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0) {
    s_max[warp] = m;
    s_sum[warp] = sum;
  }
  if (tid < NB) s_hist[tid] = 0;
  if (tid == 0) s_run = 0;
  __syncthreads();
  int mx = 0;
  long long total = 0;
  for (int q = 0; q < 32; ++q) {
    mx = max(mx, s_max[q]);
    total += s_sum[q];
  }
  // slices with more tiles than half a block's fair share are split (half:
  // a tile of a heavy slice costs more than one of a light slice, since it
  // holds more of the slice's pixel rows; at the full share the heaviest
  // slices of an 8 x 512 x 512 RGB batch stayed whole and set the end of
  // the launch, 9.9 ms against 5.5 ms for the tensor-core pass)
  const long long share = (long long)NL * total / max(2 * resident, 1);
  for (int c0 = 0; c0 < nkeys; c0 += 1024) {
    const int k = c0 + tid;
    const bool heavy = k < nkeys && cnt[k] >= 2 && (long long)cnt[k] > share;
    const unsigned bal = __ballot_sync(0xffffffffu, heavy);
    if (lane == 0) s_n[warp] = __popc(bal);
    __syncthreads();
    int rank = s_run + __popc(bal & lt), add = 0;
    for (int q = 0; q < 32; ++q) {
      rank += q < warp ? s_n[q] : 0;
      add += s_n[q];
    }
    const bool split = heavy && rank < smax;
    if (k < nkeys) slot[k] = split ? rank : -1;
    if (split) split_key[rank] = k;
    __syncthreads();
    if (tid == 0) s_run += add;
    __syncthreads();
  }
  const int nsplit = min(s_run, smax), nitems = nkeys + nsplit;
  __syncthreads();  // slot and split_key written by the block are visible
  // item id: k < nkeys is chunk 0 of key k, nkeys + r chunk 1 of split_key[r]
  auto item_key = [&](int id) { return id < nkeys ? id : split_key[id - nkeys]; };
  auto bucket = [&](int id) {
    const int key = item_key(id);
    const int nch = slot[key] >= 0 ? 2 : 1, w = (cnt[key] + nch - 1) / nch;
    return NB - 1 - (int)((long long)w * NB / ((long long)mx + 1));  // 0: the heaviest
  };
  for (int id = tid; id < nitems; id += 1024) atomicAdd(&s_hist[bucket(id)], 1);
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int b = 0; b < NB; ++b) {
      s_base[b] = run;
      run += s_hist[b];
    }
  }
  __syncthreads();
  for (int c0 = 0; c0 < nitems; c0 += 1024) {
    const int id = c0 + tid;
    const bool valid = id < nitems;
    const int b = valid ? bucket(id) : NB;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int rank = __popc(peers & lt);
    for (int i = tid; i < 32 * NB; i += 1024) (&s_wc[0][0])[i] = 0;
    __syncthreads();
    if (valid && rank == 0) s_wc[warp][b] = __popc(peers);
    __syncthreads();
    if (tid < NB) {
      int run = 0;
      for (int q = 0; q < 32; ++q) {
        const int c = s_wc[q][tid];
        s_wc[q][tid] = run;
        run += c;
      }
      s_tot[tid] = run;
    }
    __syncthreads();
    if (valid) {
      const int pos = s_base[b] + s_wc[warp][b] + rank;
      if (pos < nitems) order[pos] = item_key(id) * 2 + (id < nkeys ? 0 : 1);
    }
    __syncthreads();
    if (tid < NB) s_base[tid] += s_tot[tid];
    __syncthreads();
  }
  for (int i = nitems + tid; i < nkeys + smax; i += 1024) order[i] = -1;
}

// The end of a block whose item is one of two chunks of a split slice: its
// partial gradient is in its own slab (written by the block); after both
// chunks have written theirs, the second block to finish adds them in
// chunk order (the same sum whichever finishes last) into out.  Every
// thread of the block calls it; nt = threads of the block.
__device__ __forceinline__ void combine_chunks(const float* slab0, const float* slab1, float* out,
                                               int n, int* tick, int nt) {
  __shared__ int s_last;
  __threadfence();  // this block's partial is visible device-wide
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(tick, 1) == 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int i = threadIdx.x; i < n; i += nt) out[i] = __ldcg(slab0 + i) + __ldcg(slab1 + i);
  if (threadIdx.x == 0) *tick = 0;
}

// Block (rank * NL + lam) computes item order[rank] (a slice, or one tile
// chunk of a split slice) at wavelength lam over its tiles that use the
// slice, and writes the slice's gradient (split slices: through the two
// chunks' slabs, see combine_chunks).
template <int NT, int SPT, class TI>
__global__ void __launch_bounds__(NT, NT <= 256 ? 3 : (NT <= 320 ? 2 : 1)) render_bwd_bank_kernel(const RenderParams P,
                                                             const float* __restrict__ gout,
                                                             const unsigned* __restrict__ bm,
                                                             int words, int ntx, int nty,
                                                             BankPlan plan,
                                                             float* __restrict__ gbank) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ks = P.ks, p = (ks - 1) >> 1, ks2 = ks * ks;
  const int KU = (ks + SEG - 1) / SEG * SEG;
  const int S = TXB + ks - 1;
  const int HH = RT_Y + ks - 1 + SEG;
  constexpr int NPX = TXB * RT_Y, NSEG = NPX / SEG;
  // one thread per segment builds the segment list below
  static_assert(NT >= NSEG, "the bank-gradient block needs a thread per segment");
  // the tile lists and segment lists use full-warp ballots
  static_assert(NT % 32 == 0, "the bank-gradient block must be whole warps");
  float* halo = reinterpret_cast<float*>(smem);          // HH x S
  float2* G = reinterpret_cast<float2*>(halo + (size_t)HH * S);  // NPX (L, R)
  int* segs = reinterpret_cast<int*>(G + NPX);            // NSEG
  __shared__ int s_nseg, s_wcnt[NSEG / 32];

  const int lam = (int)(blockIdx.x % P.NL), item = plan.order[blockIdx.x / P.NL];
  if (item < 0 || (item >> 1) >= plan.nkeys) return;  // past the last item
  const int key = item >> 1, chunk = item & 1, sl = plan.slot[key], nch = sl >= 0 ? 2 : 1;
  const int tid = threadIdx.x;
  const bool two = P.Z > 1;
  const int nstrip = ks * (KU / SEG);
  // per strip and row: (L, R) sums, one packed two-lane FMA per tap (its
  // components round like fmaf)
  float2 acc[SPT][SEG];
#pragma unroll
  for (int s = 0; s < SPT; ++s)
#pragma unroll
    for (int i = 0; i < SEG; ++i) acc[s][i] = make_float2(0.f, 0.f);

  const int kw = key >> 5;
  const unsigned kbit = 1u << (key & 31);
  const int c_lo = (P.NL == P.C) ? lam : 0, c_hi = (P.NL == P.C) ? lam + 1 : P.C;
  // the tiles that use the slice, in ascending order
  __shared__ int s_list[NT], s_twc[NT / 32];
  const size_t ntiles = (size_t)P.N * nty * ntx;
  for (size_t t0 = 0; t0 < ntiles; t0 += NT)
    for (int li = 0, nlist = slice_tiles<NT>(bm, words, kw, kbit, t0, ntiles, nch, chunk, s_list,
                                             s_twc);
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
                selected(P, n, yy, xx, &k0, &t);
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
                  acc[s][uu] = __ffma2_rn(g, make_float2(img[j + uu], img[j + uu]), acc[s][uu]);
                }
              }
            }
          }
        }
      }
  // dKf[u][v] -> B[key][lam][side][ks-1-u][ks-1-v] (a split slice: the
  // chunk's slab first)
  float* out = gbank + ((size_t)key * P.NL + lam) * 2 * ks2;
  if (nch == 2 && !SD_CHECK(sl, plan.smax)) return;
  float* dst = nch == 1 ? out : plan.slab(sl, chunk, lam, P.NL, ks2);
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
      dst[o] = acc[s][uu].x;
      dst[ks2 + o] = acc[s][uu].y;
    }
  }
  if (nch == 2)
    combine_chunks(plan.slab(sl, 0, lam, P.NL, ks2), plan.slab(sl, 1, lam, P.NL, ks2), out,
                   2 * ks2, plan.tick + (size_t)sl * P.NL + lam, NT);
}

// Quadrant bank: grad_bank = for each stored element, the sum over the four
// flip classes (class x: other side, column mirrored; class y: row mirrored)
// of the per-key gradients, in a fixed order (deterministic).  n = stored
// elements, n_kl = stored slices x wavelengths.
__global__ void bank_fold_quadrant(const float* __restrict__ keyg, size_t n, int n_kl, int ks,
                                   float* __restrict__ gbank) {
  const size_t ks2 = (size_t)ks * ks;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t kl = i / (2 * ks2), rem = i - kl * 2 * ks2;
    const int side = (int)(rem / ks2), e = (int)(rem - side * ks2), a = e / ks, b = e - a * ks;
    float acc = 0.f;
    for (int f = 0; f < 4; ++f) {
      const bool mx = f & 1, my = f & 2;
      const int vs = mx ? 1 - side : side, va = my ? ks - 1 - a : a, vb = mx ? ks - 1 - b : b;
      acc += keyg[(((size_t)f * n_kl + kl) * 2 + vs) * ks2 + (size_t)va * ks + vb];
    }
    gbank[i] = acc;
  }
}

// Workspace of a bank-gradient plan: counts, split slots, order, split keys,
// tickets, then the chunk slabs of at most smax split slices (the plan is
// the last part of a workspace and smax what the rest of it holds).
struct PlanLayout {
  int smax;
  size_t cnt, slot, order, split, tick, pbuf, total;
};

inline PlanLayout plan_layout(const RenderParams& P, int smax) {
  const int nk = n_keys(P);
  PlanLayout L;
  L.smax = smax;
  size_t o = 0;
  L.cnt = o;
  o += (size_t)nk * 4;
  L.slot = o;
  o += (size_t)nk * 4;
  L.order = o;
  o += ((size_t)nk + smax) * 4;
  L.split = o;
  o += (size_t)smax * 4;
  L.tick = o;
  o += (size_t)smax * P.NL * 4;
  L.pbuf = (o + 255) & ~(size_t)255;
  o = L.pbuf + (size_t)2 * smax * P.NL * 2 * P.ks * P.ks * 4;
  L.total = (o + 255) & ~(size_t)255;
  return L;
}

// split slots a full workspace provides: an eighth of the keys, at least 32
inline int plan_smax(const RenderParams& P) { return std::max(32, n_keys(P) / 8); }
inline size_t plan_bytes(const RenderParams& P) { return plan_layout(P, plan_smax(P)).total; }

// the most split slots (up to plan_smax) whose plan fits in avail bytes; -1
// if not even a plan without splits fits
inline int plan_smax_fit(const RenderParams& P, size_t avail) {
  const size_t per = (size_t)2 * P.NL * 2 * P.ks * P.ks * 4 + (size_t)(2 + P.NL) * 4;
  const size_t base = plan_layout(P, 0).total;
  if (avail < base) return -1;
  int sm = (int)std::min<size_t>((size_t)plan_smax(P), (avail - base) / per);
  while (sm > 0 && plan_layout(P, sm).total > avail) --sm;
  return sm;
}

// blocks of kernel fn (nt threads, smem bytes) resident on the whole GPU
inline sd_status resident_blocks(const void* fn, int nt, size_t smem, int* out) {
  int dev = 0, sms = 0, nb = 0;
  SD_CUDA_TRY(cudaGetDevice(&dev));
  SD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, nt, smem));
  *out = std::max(1, nb) * std::max(1, sms);
  return SD_OK;
}

// Builds the plan in ws (plan_layout(P, smax).total bytes, 256-byte
// aligned) for a bank kernel of which `resident` blocks run at once; returns
// it in *plan and the number of block ranks (items) to launch in *ranks.
inline sd_status launch_plan(const RenderParams& P, const unsigned* bm, int words, size_t ntiles,
                             int resident, void* ws, int smax, BankPlan* plan, int* ranks,
                             cudaStream_t s) {
  const PlanLayout L = plan_layout(P, smax);
  const int nk = n_keys(P);
  char* b = reinterpret_cast<char*>(ws);
  int* cnt = reinterpret_cast<int*>(b + L.cnt);
  int* slot = reinterpret_cast<int*>(b + L.slot);
  int* order = reinterpret_cast<int*>(b + L.order);
  int* split = reinterpret_cast<int*>(b + L.split);
  int* tick = reinterpret_cast<int*>(b + L.tick);
  SD_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)nk * 4, s));
  if (L.smax > 0) SD_CUDA_TRY(cudaMemsetAsync(tick, 0, (size_t)L.smax * P.NL * 4, s));
  dim3 g(words, (unsigned)((ntiles + 1023) / 1024));
  slice_count_kernel<<<g, 256, 0, s>>>(bm, words, ntiles, nk, cnt);
  sd_status st = launch_status();
  if (st != SD_OK) return st;
  slice_order_kernel<<<1, 1024, 0, s>>>(cnt, nk, P.NL, resident, L.smax, slot, split, order);
  st = launch_status();
  if (st != SD_OK) return st;
  plan->order = order;
  plan->slot = slot;
  plan->tick = tick;
  plan->pbuf = reinterpret_cast<float*>(b + L.pbuf);
  plan->nkeys = nk;
  plan->smax = L.smax;
  *ranks = nk + L.smax;
  return SD_OK;
}

template <int NT, int SPT, class TI>
sd_status launch_bank_bwd(const RenderParams& P, const float* gout, const unsigned* bm, int words,
                          int ntx, int nty, void* plan_ws, int smax, float* gbank,
                          float* quad_buf, cudaStream_t s) {
  const int ks = P.ks;
  size_t smem = (size_t)(RT_Y + ks - 1 + SEG) * (TXB + ks - 1) * 4 + (size_t)TXB * RT_Y * 8 +
                (size_t)(TXB * RT_Y / SEG) * 4;
  auto k = render_bwd_bank_kernel<NT, SPT, TI>;
  SD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int resident = 0, ranks = 0;
  sd_status st = resident_blocks(reinterpret_cast<const void*>(k), NT, smem, &resident);
  if (st != SD_OK) return st;
  BankPlan plan;
  st = launch_plan(P, bm, words, (size_t)P.N * ntx * nty, resident, plan_ws, smax, &plan, &ranks,
                   s);
  if (st != SD_OK) return st;
  // a quadrant bank's gradients are per key (flip class) first, then folded
  const bool quad = P.fmode == SD_FIELD_QUADRANT;
  k<<<(unsigned)ranks * P.NL, NT, smem, s>>>(P, gout, bm, words, ntx, nty, plan,
                                             quad ? quad_buf : gbank);
  st = launch_status();
  if (st != SD_OK || !quad) return st;
  const size_t n = (size_t)P.FC * P.Z * P.NL * 2 * ks * ks;
  bank_fold_quadrant<<<1024, 256, 0, s>>>(quad_buf, n, P.FC * P.Z * P.NL, ks, gbank);
  return launch_status();
}

constexpr size_t SMEM_CAP_B = 227 * 1024;

inline size_t bitmap_bytes(int N, int tx, int ty, int nkeys) {
  return ((size_t)N * tx * ty * bitmap_words(nkeys) * 4 + 255) & ~(size_t)255;
}
// per-key gradient slab of a quadrant bank (its keys carry 4 flip classes)
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

// The per-pixel selection table of the call, written once.
inline sd_status launch_select_table(const RenderParams& P, int2* sel, cudaStream_t s) {
  const size_t npx = (size_t)P.N * P.H * P.W;
  const int blocks = (int)std::min<size_t>((npx + 255) / 256, (size_t)152 * 16);
  select_table_kernel<<<blocks, 256, 0, s>>>(P, sel);
  return launch_status();
}

// The image gradient: bank re-layout, then one launch per
// phase of non-overlapping strips (phase order fixed: deterministic).
template <class TB>
sd_status launch_img_bwd(const RenderParams& P, const float* gout, float* gaif, void* ws,
                         cudaStream_t s) {
  const ImgLayout IL = img_layout(P);
  char* base = reinterpret_cast<char*>(ws);
  const int2* sel = P.sel;
  float* kcol = reinterpret_cast<float*>(base);
  unsigned short* ext = reinterpret_cast<unsigned short*>(base + IL.kcol_bytes);
  sd_status st;
  const int n_kl = n_keys(P) * P.NL;
  const size_t ksm = (size_t)2 * P.ks * P.ks * 4;
  SD_CUDA_TRY(cudaFuncSetAttribute(kernel_columns_kernel<TB>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ksm));
  kernel_columns_kernel<TB><<<n_kl, 256, ksm, s>>>(P, IL, kcol, ext);
  st = launch_status();
  if (st != SD_OK) return st;
  const int nrange = (P.W + IG_SW - 1) / IG_SW, nrb = (P.H + 7) / 8;
  const bool wide = P.ks > 65;
  const size_t smem =
      (size_t)IG_NW * (8 * IG_SW * 16 + 2 * (8 * (wide ? 192 : 128) + 16) * 4);
  auto k = wide ? render_bwd_img_kernel<192> : render_bwd_img_kernel<128>;
  SD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int phase = 0; phase < IL.nphase && phase < nrange; ++phase) {
    const int nr_phase = (nrange - phase + IL.nphase - 1) / IL.nphase;
    const long long grid = (long long)nr_phase * nrb * P.N * P.C;  // one item per block
    if (grid > 0x7fffffffll) return SD_ERR_UNSUPPORTED;
    k<<<(unsigned)grid, IG_NW * 32, smem, s>>>(P, IL, gout, sel, kcol, ext, phase, nr_phase,
                                               nrb, gaif);
    st = launch_status();
    if (st != SD_OK) return st;
  }
  return SD_OK;
}

template <class TI>
sd_status launch_bank_bwd_any(const RenderParams& P, const float* gout, const unsigned* bm,
                              int words, int tx, int ty, void* plan_ws, int smax,
                              float* gbank, float* quad_buf, cudaStream_t s) {
  int KU = (P.ks + SEG - 1) / SEG * SEG;
  int nstrip = P.ks * (KU / SEG);
  // where the strips fill 512-640 slots (ks = 61..65): 320 threads with two
  // strips each, two blocks per SM, so that one block's staging of a tile
  // overlaps the other's products (608 threads x 1 strip, one block per SM,
  // was 1.5 % slower; 256 threads x 3 strips left a quarter of the slots idle)
  if (nstrip > 512 && nstrip <= 640)
    return launch_bank_bwd<320, 2, TI>(P, gout, bm, words, tx, ty, plan_ws, smax, gbank, quad_buf,
                                       s);
  if (nstrip <= 256 * 3)
    return launch_bank_bwd<256, 3, TI>(P, gout, bm, words, tx, ty, plan_ws, smax, gbank, quad_buf,
                                       s);
  return launch_bank_bwd<512, 4, TI>(P, gout, bm, words, tx, ty, plan_ws, smax, gbank, quad_buf,
                                       s);
}


// ---------------------------------------------------------------------------
// 4. bank gradient on the tensor cores (BF16 or FP16 image; the weighted
// gradients w * G rounded to the image's type; FP32 accumulation in tensor
// memory)
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
constexpr uint32_t BG_DRAIN = 1u << 24;  // final wait for the CTA's own products

__host__ __device__ inline int bg_nug(int ks) { return (ks + 15) / 16; }
__host__ __device__ inline size_t bg_img_bytes(int ks) {
  return ((size_t)(RT_Y + 16 * bg_nug(ks)) * BG_IWB + 127) / 128 * 128;
}
__host__ __device__ inline size_t bg_smem(int ks) {
  return bg_img_bytes(ks) + (size_t)2 * RT_Y * BG_GW * 2 + (size_t)BG_NB * BG_BBUF;
}

__device__ __forceinline__ bool bg_wait(uint64_t* bar, uint32_t parity, int* err,
                                        uint32_t limit) {
  if (tc::mbar_wait(bar, parity, limit, err)) return true;
  atomicExch(err, 1);
  return false;
}

template <bool F16>
__global__ void __launch_bounds__(BG_NT, 2) bank_grad_tc_kernel(
    const RenderParams P, const float* __restrict__ gout, const unsigned* __restrict__ bm,
    int words, int ntx, int nty, BankPlan plan, float* __restrict__ gbank, int* err,
    uint32_t wlim) {
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
  // block (rank * NL + lam): item order[rank] (a slice or one tile chunk of
  // a split slice; the items with the most tiles first)
  const int lam = (int)(blockIdx.x % P.NL), item = plan.order[blockIdx.x / P.NL];
  if (item < 0 || (item >> 1) >= plan.nkeys) return;  // past the last item
  const int key = item >> 1, chunk = item & 1, sl = plan.slot[key], nch = sl >= 0 ? 2 : 1;
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
  const uint32_t idesc = F16 ? tc::idesc_f16_f32(128, BG_N) : tc::idesc_bf16_f32(128, BG_N);
  const uint32_t img_a = tc::smem_u32(img), ring_a = tc::smem_u32(bring);
  int c_row = 0, visits = 0;
  unsigned inited = 0;  // kernel-row groups written (MMA thread)
  bool issuing = true;  // MMA thread: false from the first wait that gave up

  // the tiles that use the slice, in ascending order
  __shared__ int s_list[BG_NT], s_twc[BG_NT / 32];
  const size_t ntiles = (size_t)P.N * nty * ntx;
  for (size_t t0 = 0; t0 < ntiles; t0 += BG_NT)
    for (int li = 0, nlist = slice_tiles<BG_NT>(bm, words, kw, kbit, t0, ntiles, nch, chunk,
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
            if (lane == 0) bg_wait(&s_tile, (uint32_t)(visits - 1) & 1u, err, wlim);
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
            int2 sq[BG_PPR];
            float gq[BG_PPR][2];
#pragma unroll
            for (int t = 0; t < BG_PPR; ++t) {
              const int i = tid + (t0 + t) * BG_NT, r = i / TXB, x = i - r * TXB;
              const int yy = y0 + r, xx = x0 + x;
              const bool in = yy < P.H && xx < P.W;
              const size_t o = (size_t)yy * P.W + xx;
              sq[t] = in ? P.sel[(size_t)n * P.H * P.W + o] : make_int2(-1, 0);
              gq[t][0] = in ? goL[o] : 0.f;
              gq[t][1] = in ? goR[o] : 0.f;
            }
#pragma unroll
            for (int t = 0; t < BG_PPR; ++t) {
              const int i = tid + (t0 + t) * BG_NT, r = i / TXB, x = i - r * TXB;
              const int yy = y0 + r, xx = x0 + x;
              float gl = 0.f, gr = 0.f;
              if (yy < P.H && xx < P.W) {
                const int k0 = sq[t].x;
                const float tt = __int_as_float(sq[t].y);
                const float w = (k0 == key) ? (two ? 1.f - tt : 1.f)
                                            : ((two && k0 + 1 == key) ? tt : 0.f);
                gl = w * gq[t][0];
                gr = w * gq[t][1];
              }
              const unsigned short bl = tc::to_op16(gl, F16);
              const unsigned short br = tc::to_op16(gr, F16);
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
                if (lane == 0) bg_wait(&s_empty[b], (uint32_t)(cg / BG_NB - 1) & 1u, err, wlim);
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
              for (int k = 0; k < nrow && issuing; ++k) {
                const int cg = c_row + k, b = cg % BG_NB;
                issuing = bg_wait(&s_full[b], (uint32_t)(cg / BG_NB) & 1u, err, wlim);
                if (!issuing) break;
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
  // every MMA has completed; the accumulator holds the block's gradient.
  // This drain is bounded but not cut short by the error flag, so that no
  // product is still running when the tensor memory is read and freed.
  if (tid == 0) {
    tc::commit(&s_done);
    s_init = (int)inited;
  }
  if (lane == 0 && !tc::mbar_wait(&s_done, 0, BG_DRAIN)) atomicExch(err, 1);
  __syncwarp();
  __syncthreads();
  tc::fence_after_sync();
  const int ks2 = ks * ks;
  float* out = gbank + ((size_t)key * P.NL + lam) * 2 * ks2;
  float* dst = nch == 1 ? out : plan.slab(sl, chunk, lam, P.NL, ks2);
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
          const long long o = (long long)side * ks2 + (long long)(ks - 1 - u) * ks + (ks - 1 - vv);
          if (vv < ks && SD_CHECK(o, 2 * ks2)) dst[o] = ((ini >> ug) & 1u) ? v[side * 16 + i] : 0.f;
        }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 256);
  if (nch == 2)
    combine_chunks(plan.slab(sl, 0, lam, P.NL, ks2), plan.slab(sl, 1, lam, P.NL, ks2), out,
                   2 * ks2, plan.tick + (size_t)sl * P.NL + lam, BG_NT);
}

sd_status launch_bank_grad_tc(const RenderParams& P, const float* gout, const unsigned* bm,
                              int words, int ntx, int nty, void* plan_ws, int smax,
                              float* gbank, float* quad_buf, int* err, bool f16,
                              cudaStream_t s) {
  const int ks = P.ks;
  // at least 80 KB: two CTAs per SM, the tensor memory's 512 columns
  const size_t smem = std::max(bg_smem(ks), (size_t)80 * 1024);
  auto k = f16 ? bank_grad_tc_kernel<true> : bank_grad_tc_kernel<false>;
  SD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int resident = 0, ranks = 0;
  sd_status st = resident_blocks(reinterpret_cast<const void*>(k), BG_NT, smem, &resident);
  if (st != SD_OK) return st;
  BankPlan plan;
  st = launch_plan(P, bm, words, (size_t)P.N * ntx * nty, resident, plan_ws, smax, &plan, &ranks,
                   s);
  if (st != SD_OK) return st;
  const bool quad = P.fmode == SD_FIELD_QUADRANT;
  k<<<(unsigned)ranks * P.NL, BG_NT, smem, s>>>(P, gout, bm, words, ntx, nty, plan,
                                                quad ? quad_buf : gbank, err,
                                                wait_limit(BG_WAIT));
  st = launch_status();
  if (st != SD_OK || !quad) return st;
  const size_t n = (size_t)P.FC * P.Z * P.NL * 2 * ks * ks;
  bank_fold_quadrant<<<1024, 256, 0, s>>>(quad_buf, n, P.FC * P.Z * P.NL, ks, gbank);
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
  *bytes = sel_table_bytes(P) + img_layout(P).total + bitmap_bytes(N, tx, ty, n_keys(P)) +
           (P.fmode == SD_FIELD_QUADRANT ? bank_bytes(P) : 0) + plan_bytes(P);
  return SD_OK;
}

sd_status sd_dp_render_backward(const float* grad_out, const void* aif, const float* depth_m,
                                const void* bank, const sd_bank_layout* layout, int N, int C,
                                int H, int W, int image_dtype, float* grad_aif,
                                float* grad_bank, void* workspace, size_t workspace_bytes,
                                void* stream) {
  SD_API_RANGE("sd_dp_render_backward");
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
  if (!grad_aif && !grad_bank) return SD_OK;
  // the selection table comes first; both passes read it
  const size_t sel_bytes = sel_table_bytes(P);
  if (!workspace || workspace_bytes < sel_bytes ||
      (reinterpret_cast<uintptr_t>(workspace) & 255))
    return SD_ERR_ARG;
  int2* sel = reinterpret_cast<int2*>(workspace);
  P.sel = sel;
  workspace = reinterpret_cast<char*>(workspace) + sel_bytes;
  workspace_bytes -= sel_bytes;
  // then the image pass's tables
  const size_t img_bytes = grad_aif ? img_layout(P).total : 0;
  if (grad_aif && workspace_bytes < img_bytes) return SD_ERR_ARG;
  // then the bank pass's bitmap, a quadrant bank's per-key slab (folded
  // onto the stored quadrant) and the work plan, whose split slots take
  // what the rest of the workspace holds
  int smax = 0;
  if (grad_bank) {
    int tx, ty;
    bwd_tiles(H, W, &tx, &ty);
    const size_t fixed = img_bytes + bitmap_bytes(N, tx, ty, n_keys(P)) +
                         (P.fmode == SD_FIELD_QUADRANT ? bank_bytes(P) : 0);
    if (workspace_bytes < fixed) return SD_ERR_ARG;
    smax = plan_smax_fit(P, workspace_bytes - fixed);
    if (smax < 0) return SD_ERR_ARG;
  }
  st = launch_select_table(P, sel, s);
  if (st != SD_OK) return st;
  if (grad_aif) {
    SD_CUDA_TRY(cudaMemsetAsync(grad_aif, 0, (size_t)N * C * H * W * 4, s));
    // the re-layout reads the bank in its storage type
    const int bt = layout->dtype;
    sd_status r = bt == SD_F32 ? launch_img_bwd<float>(P, grad_out, grad_aif, workspace, s)
                  : bt == SD_BF16
                      ? launch_img_bwd<__nv_bfloat16>(P, grad_out, grad_aif, workspace, s)
                      : launch_img_bwd<__half>(P, grad_out, grad_aif, workspace, s);
    if (r != SD_OK) return r;
    workspace = reinterpret_cast<char*>(workspace) + img_bytes;
    workspace_bytes -= img_bytes;
  }
  if (grad_bank) {
    int tx, ty;
    bwd_tiles(H, W, &tx, &ty);
    size_t words = bitmap_words(n_keys(P));
    size_t need = bitmap_bytes(N, tx, ty, n_keys(P));
    unsigned* bm = reinterpret_cast<unsigned*>(workspace);
    float* quad_buf = reinterpret_cast<float*>(reinterpret_cast<char*>(workspace) + need);
    void* plan_ws = reinterpret_cast<char*>(workspace) + need +
                    (P.fmode == SD_FIELD_QUADRANT ? bank_bytes(P) : 0);
    dim3 g1(tx, ty, N);
    slice_bitmap_kernel<<<g1, NT_BM, words * 4, s>>>(P, bm, (int)words);
    sd_status r = launch_status();
    if (r != SD_OK) return r;
    // the bank pass reads the image in its storage type
    r = image_dtype == SD_F32
            ? launch_bank_bwd_any<float>(P, grad_out, bm, (int)words, tx, ty, plan_ws, smax,
                                         grad_bank, quad_buf, s)
        : image_dtype == SD_BF16
            ? launch_bank_bwd_any<__nv_bfloat16>(P, grad_out, bm, (int)words, tx, ty, plan_ws,
                                                 smax, grad_bank, quad_buf, s)
            : launch_bank_bwd_any<__half>(P, grad_out, bm, (int)words, tx, ty, plan_ws, smax,
                                          grad_bank, quad_buf, s);
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
  *bytes = 256 + sel_table_bytes(P) + bitmap_bytes(N, tx, ty, n_keys(P)) +
           (P.fmode == SD_FIELD_QUADRANT ? bank_bytes(P) : 0) + plan_bytes(P);
  return SD_OK;
}

sd_status sd_dp_render_bank_grad_tc(const float* grad_out, const void* aif, const float* depth_m,
                                    const sd_bank_layout* layout, int N, int C, int H, int W,
                                    int image_dtype, float* grad_bank, void* workspace,
                                    size_t workspace_bytes, void* stream) {
  SD_API_RANGE("sd_dp_render_bank_grad_tc");
  using namespace sd;
  if (!grad_out || !aif || !depth_m || !grad_bank) return SD_ERR_ARG;
  RenderParams P;
  sd_status st = setup_bwd(layout, N, C, H, W, P);
  if (st != SD_OK) return st;
  if (image_dtype != SD_BF16 && image_dtype != SD_F16) return SD_ERR_UNSUPPORTED;
  // the epilogue maps kernel columns 0..64 (8 column groups x 8 shifts and
  // one more): ks <= 65
  if (P.ks > 65 || bg_smem(P.ks) > 227 * 1024) return SD_ERR_UNSUPPORTED;
  P.aif = aif;
  P.depth = depth_m;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t bank_elems = (size_t)P.FC * P.Z * P.NL * 2 * P.ks * P.ks;
  int tx, ty;
  bwd_tiles(H, W, &tx, &ty);
  const size_t words = bitmap_words(n_keys(P));
  const size_t sel_bytes = sel_table_bytes(P);
  const int nk = n_keys(P);
  const size_t need = 256 + sel_bytes + bitmap_bytes(N, tx, ty, nk);
  const size_t quad_bytes = P.fmode == SD_FIELD_QUADRANT ? bank_bytes(P) : 0;
  if (!workspace || workspace_bytes < need + quad_bytes ||
      (reinterpret_cast<uintptr_t>(workspace) & 255))
    return SD_ERR_ARG;
  const int smax = plan_smax_fit(P, workspace_bytes - need - quad_bytes);
  if (smax < 0) return SD_ERR_ARG;
  int* err = reinterpret_cast<int*>(workspace);
  SD_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  if (N == 0 || H == 0 || W == 0) {
    SD_CUDA_TRY(cudaMemsetAsync(grad_bank, 0, bank_elems * 4, s));
    return SD_OK;
  }
  int2* sel = reinterpret_cast<int2*>(reinterpret_cast<char*>(workspace) + 256);
  P.sel = sel;
  unsigned* bm = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(workspace) + 256 + sel_bytes);
  float* quad_buf = reinterpret_cast<float*>(reinterpret_cast<char*>(workspace) + need);
  void* plan_ws = reinterpret_cast<char*>(workspace) + need + quad_bytes;
  st = launch_select_table(P, sel, s);
  if (st != SD_OK) return st;
  dim3 g1(tx, ty, N);
  slice_bitmap_kernel<<<g1, NT_BM, words * 4, s>>>(P, bm, (int)words);
  st = launch_status();
  if (st != SD_OK) return st;
  return launch_bank_grad_tc(P, grad_out, bm, (int)words, tx, ty, plan_ws, smax, grad_bank,
                             quad_buf, err, image_dtype == SD_F16, s);
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
// device pointer).  Kept for the process's life: a cudaDeviceReset would
// move the array, which the header excludes.
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
                                                   const float* depth_m, const void* bank,
                                                   const sd_bank_layout* layout, int N, int C,
                                                   int H, int W, float* grad_aif,
                                                   float* grad_bank, void* stream) {
  SD_API_RANGE("sd_dp_render_backward_noalloc");
  using namespace sd;
  void* ws = nullptr;
  size_t need = 0;
  if (grad_aif || grad_bank) {
    // the selection table, the image pass's tables and the bank pass's
    // bitmap, a quadrant bank's per-key slab and a work plan without split
    // slots must fit (split slots take what the array holds beyond that)
    RenderParams P;
    sd_status st = setup_bwd(layout, N, C, H, W, P);
    if (st != SD_OK) return st;
    int tx, ty;
    bwd_tiles(H, W, &tx, &ty);
    need = sel_table_bytes(P);
    if (grad_aif) need += img_layout(P).total;
    if (grad_bank)
      need += bitmap_bytes(N, tx, ty, n_keys(P)) + plan_layout(P, 0).total +
              (P.fmode == SD_FIELD_QUADRANT ? bank_bytes(P) : 0);
    if (need > NOALLOC_SCRATCH_BYTES) return SD_ERR_CAPACITY;
    st = noalloc_scratch(&ws);
    if (st != SD_OK) return st;
  }
  return sd_dp_render_backward(grad_out, aif, depth_m, bank, layout, N, C, H, W, SD_F32,
                               grad_aif, grad_bank, ws, NOALLOC_SCRATCH_BYTES, stream);
}

SD_CHECK_TU(render_bwd)
