// Definitions shared by the render forward and backward kernels.
#pragma once

#include <cstring>

#include "common.cuh"

namespace sd {

constexpr int SEG = 8;          // rows per segment (one lane's pixels)
constexpr int RT_Y = 32;        // tile height (rows)
constexpr int RK = 256;         // slice keys per window
constexpr int MAX_CHUNKS = 512;   // >= NT*2*SEG/32 + RK for NT <= 512

struct RenderParams {
  const void* aif;
  const float* depth;
  const void* bank;
  void* out;
  const int2* sel;  // backward passes: per-pixel (key, t bits), [N][H][W]
  int N, C, H, W;
  int F, Z, NL, ks;
  int fmode;       // SD_FIELD_RADIAL or SD_FIELD_QUADRANT
  int FC;          // field cells of the bank: F (radial) or F * F (quadrant)
  float pitch;
  int halo_w;      // row stride of the staged tile (floats)
  int halo_h;
  float fh[SD_MAX_BANK_FIELDS];
  float iq[SD_MAX_BANK_DEPTHS];  // 1.0f / depth_m[j] (strictly descending)
};

// nearest of the F ascending heights fh to r (ties to the lower index),
// clamped at both ends
__device__ __forceinline__ int nearest_field(const float* fh, int F, float r) {
  if (r <= fh[0]) return 0;
  if (r >= fh[F - 1]) return F - 1;
  int a = 0, b = F - 1;  // fh[a] <= r < fh[b]
  while (b - a > 1) {
    int m = (a + b) >> 1;
    if (fh[m] <= r) a = m; else b = m;
  }
  float dlo = __fsub_rn(r, fh[a]);
  float dhi = __fsub_rn(fh[a + 1], r);
  return (dhi < dlo) ? a + 1 : a;
}

// Per-pixel bank selection in FP32 without contraction (the same sequence of
// IEEE operations as the oracle's selection).  The key is f * Z + z0 with f
// the field cell; in quadrant mode f = flips * F * F + fx * F + fy, flips =
// (X < 0) + 2 (Y < 0), so that key + 1 is still the next depth slice.
__device__ __forceinline__ void select_slice(const RenderParams& P, int row, int col,
                                             float depth, int* key, float* t) {
  float X = __fmul_rn(__fsub_rn((float)col, 0.5f * (float)(P.W - 1)), P.pitch);
  float Y = __fmul_rn(__fsub_rn((float)row, 0.5f * (float)(P.H - 1)), P.pitch);
  int F = P.F, f;
  if (P.fmode == SD_FIELD_QUADRANT) {
    const int fx = nearest_field(P.fh, F, fabsf(X)), fy = nearest_field(P.fh, F, fabsf(Y));
    const int flips = (X < 0.f ? 1 : 0) + (Y < 0.f ? 2 : 0);
    f = flips * P.FC + fx * F + fy;
  } else {
    float rho = __fsqrt_rn(__fadd_rn(__fmul_rn(X, X), __fmul_rn(Y, Y)));
    f = nearest_field(P.fh, F, rho);
  }
  int Z = P.Z, z0;
  float tt;
  if (Z == 1) {
    z0 = 0;
    tt = 0.f;
  } else {
    float q = __fdiv_rn(1.0f, depth);
    if (q >= P.iq[0]) {
      z0 = 0;
      tt = 0.f;
    } else if (q <= P.iq[Z - 1]) {
      z0 = Z - 2;
      tt = 1.f;
    } else {
      int a = 0, b = Z - 1;  // iq[a] >= q > iq[b]
      while (b - a > 1) {
        int m = (a + b) >> 1;
        if (P.iq[m] >= q) a = m; else b = m;
      }
      z0 = a;
      tt = __fdiv_rn(__fsub_rn(P.iq[a], q), __fsub_rn(P.iq[a], P.iq[a + 1]));
    }
  }
  *key = f * Z + z0;
  *t = tt;
}

// The selection of pixel (n, row, col) from the per-pixel table that the
// backward passes build once per call (select_slice's result, bit for bit).
__device__ __forceinline__ void selected(const RenderParams& P, int n, int row, int col,
                                         int* key, float* t) {
  const int2 v = P.sel[((size_t)n * P.H + row) * P.W + col];
  *key = v.x;
  *t = __int_as_float(v.y);
}

// Keys select_slice can produce: field cells x depths, times 4 flip classes
// for a quadrant bank.
inline int n_keys(const RenderParams& P) {
  return P.FC * P.Z * (P.fmode == SD_FIELD_QUADRANT ? 4 : 1);
}

inline sd_status check_layout(const sd_bank_layout* L, RenderParams& P) {
  if (!L || !L->field_h_mm || !L->depths_m) return SD_ERR_ARG;
  if (L->n_field < 1 || L->n_field > SD_MAX_BANK_FIELDS || L->n_depth < 1 ||
      L->n_depth > SD_MAX_BANK_DEPTHS || L->n_lambda < 1)
    return SD_ERR_ARG;
  if (L->ks < 1 || !(L->ks & 1)) return SD_ERR_ARG;
  if (L->ks > 127) return SD_ERR_UNSUPPORTED;
  if (!(L->pitch_mm > 0)) return SD_ERR_ARG;
  for (int i = 0; i < L->n_field; ++i) {
    P.fh[i] = L->field_h_mm[i];
    if (i && !(P.fh[i] > P.fh[i - 1])) return SD_ERR_ARG;
  }
  for (int j = 0; j < L->n_depth; ++j) {
    if (!(L->depths_m[j] > 0)) return SD_ERR_ARG;
    P.iq[j] = 1.0f / L->depths_m[j];
    if (j && !(L->depths_m[j] > L->depths_m[j - 1])) return SD_ERR_ARG;
  }
  if (L->field_mode != SD_FIELD_RADIAL && L->field_mode != SD_FIELD_QUADRANT) return SD_ERR_ARG;
  if (L->field_mode == SD_FIELD_QUADRANT && !(L->field_h_mm[0] >= 0.f)) return SD_ERR_ARG;
  P.fmode = L->field_mode;
  P.F = L->n_field;
  P.FC = P.fmode == SD_FIELD_QUADRANT ? P.F * P.F : P.F;
  P.Z = L->n_depth;
  P.NL = L->n_lambda;
  P.ks = L->ks;
  P.pitch = L->pitch_mm;
  return SD_OK;
}

}  // namespace sd
