// Lens table, paraxial set-up and the DP PSF trace kernels (sm_103a).
//
// Sec. 3.1 of He et al. (ICCV 2025): a ray set A from the object point p to
// N x N entrance-pupil samples is refracted surface by surface (Snell's law)
// to the sensor plane; each landing point O_k with direction D_k is assigned
// to the left or right sub-pixel of its DP pixel with the boundary lines of
// Eq. (1) (inside the microlens) or Eq. (2) (outside), and PSF_L / PSF_R
// accumulate unit ray energies (Eq. 3), then are sum-normalised (Sec. 3.2).
//
// GPU design: one thread per ray, the lens prescription in __constant__
// memory (uniform across a warp), one thread block per PSF request with the
// [2][ks][ks] patch in shared memory.  Hard binning uses warp-aggregated
// shared-memory integer atomics (__match_any_sync on the destination bin);
// no global atomics.  The per-request paraxial set-up (entrance pupil,
// object point, refractive indices at the request wavelength) runs in FP64
// in the block prologue; the per-ray trace is FP32.

#define SD_TU 1  // translation unit id of this file's SD_CHECK sites
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include <type_traits>

#include "common.cuh"

namespace sd {

// ---------------------------------------------------------------------------
// Device lens image
// ---------------------------------------------------------------------------
struct DevSurf {
  float c, k;       // curvature (1/mm) and conic
  float a[5];       // a4..a12
  float da[5];      // (m) * a_2m: derivative coefficients of the sag in u = rho^2
  float t;          // thickness after the surface (mm); last: sensor distance
  float sd2;        // clear semi-diameter squared
  int type;         // SD_SURF_REFRACT / SD_SURF_STOP
  int asph;         // any a_2m != 0 -> Newton refinement
  int flat;         // c == 0 -> plane start
  int kind;         // bits: 1 refracting, 2 asphere, 4 flat (one load)
};

enum { K_REFRACT = 1, K_ASPH = 2, K_FLAT = 4 };

struct DevLens {
  int n, stop;
  double z_front;   // most negative z of surface 0 inside its aperture
  double sd_stop;
  double c[SD_MAX_SURFACES], t[SD_MAX_SURFACES];
  double A[SD_MAX_SURFACES], B[SD_MAX_SURFACES];  // Cauchy n = A + B/lam^2 (um)
  int type[SD_MAX_SURFACES];
  DevSurf s[SD_MAX_SURFACES];
};

__constant__ DevLens c_lens[SD_MAX_LENSES];

// ---------------------------------------------------------------------------
// Paraxial optics (FP64), shared by host and device code
// ---------------------------------------------------------------------------
struct PYU {
  double y, u, n;
};

__host__ __device__ inline double cauchy(double A, double B, double lam_um) {
  return A + B / (lam_um * lam_um);
}

// y-nu trace of a ray given at the vertex plane of surface `from` (before it
// refracts) through surfaces [from, to); ends at the vertex plane of `to`.
// nlam[s] is the index after surface s at the working wavelength.
__host__ __device__ inline PYU parax(const DevLens& L, const double* nlam,
                                     double y, double u, int from, int to) {
  double n = from > 0 ? nlam[from - 1] : 1.0;
  for (int s = from; s < to; ++s) {
    double n2 = nlam[s];
    if (L.type[s] == SD_SURF_REFRACT) u = (n * u - y * (n2 - n) * L.c[s]) / n2;
    n = n2;
    y = y + L.t[s] * u;
  }
  PYU r;
  r.y = y;
  r.u = u;
  r.n = n;
  return r;
}

struct RayGen {
  double m;        // chief-ray magnification onto the sensor plane
  double x_o;      // object height (mm), object at z = -depth
  double z_ep, r_ep;
  double z_start;  // plane where rays start
};

// Entrance pupil = paraxial image of the stop in object space; object height
// from the paraxial chief ray (through the pupil centre) landing at h on the
// sensor plane.
__host__ __device__ inline RayGen ray_gen(const DevLens& L, const double* nlam,
                                          double h_mm, double depth_mm) {
  RayGen g;
  PYU a = parax(L, nlam, 1.0, 0.0, 0, L.stop);
  PYU b = parax(L, nlam, 0.0, 1.0, 0, L.stop);
  g.z_ep = b.y / a.y;
  g.r_ep = fabs(L.sd_stop / a.y);
  double u0 = -1.0 / (g.z_ep + depth_mm);
  PYU c = parax(L, nlam, 1.0 + u0 * depth_mm, u0, 0, L.n);
  g.m = c.y;
  g.x_o = h_mm / c.y;
  g.z_start = (g.z_ep <= L.z_front) ? g.z_ep : L.z_front - 1.0;
  return g;
}

__host__ __device__ inline void indices_at(const DevLens& L, double lam_nm, double* nlam) {
  double lam = lam_nm * 1e-3;
  for (int s = 0; s < L.n; ++s) nlam[s] = cauchy(L.A[s], L.B[s], lam);
}

// image distance after the last vertex for an axial object at depth d
inline double image_distance(const DevLens& L, const double* nlam, double d) {
  PYU r = parax(L, nlam, 1.0, 1.0 / d, 0, L.n - 1);
  int s = L.n - 1;
  double n2 = nlam[s], u = r.u;
  if (L.type[s] == SD_SURF_REFRACT) u = (r.n * r.u - r.y * (n2 - r.n) * L.c[s]) / n2;
  return -r.y / u;
}

}  // namespace sd

// ---------------------------------------------------------------------------
// Host lens object
// ---------------------------------------------------------------------------
struct sd_lens {
  int slot;
  int device;
  sd::DevLens img;
};

namespace sd {
namespace {

std::mutex g_mu;
bool g_used[SD_MAX_LENSES];

void cauchy_fit(double nd, double vd, double* A, double* B) {
  if (vd <= 0.0 || nd == 1.0) {
    *A = nd;
    *B = 0.0;
    return;
  }
  const double lF = 0.4861327, lC = 0.6562725, ld = 0.5875618;  // um
  *B = (nd - 1.0) / vd / (1.0 / (lF * lF) - 1.0 / (lC * lC));
  *A = nd - *B / (ld * ld);
}

bool fin(double v) { return std::isfinite(v); }

// fills the FP32 view of surface s from the FP64 parameters
void refresh_surface(DevLens& L, int s, const double* k, const double* a,
                     double sd) {
  DevSurf& d = L.s[s];
  d.c = (float)L.c[s];
  d.k = (float)k[0];
  bool asph = false;
  for (int j = 0; j < 5; ++j) {
    d.a[j] = (float)a[j];
    d.da[j] = (float)((j + 2) * a[j]);
    asph |= (a[j] != 0.0);
  }
  d.t = (float)L.t[s];
  d.sd2 = (float)(sd * sd);
  d.type = L.type[s];
  d.asph = (d.type == SD_SURF_REFRACT) && asph;
  d.flat = (d.type == SD_SURF_STOP) || (L.c[s] == 0.0);
  d.kind = (d.type == SD_SURF_REFRACT ? K_REFRACT : 0) | (d.asph ? K_ASPH : 0) |
           (d.flat ? K_FLAT : 0);
}

double sag_at(double c, double k, const double* a, double rho) {
  double u = rho * rho;
  double arg = 1.0 - (1.0 + k) * c * c * u;
  if (arg < 0) arg = 0;
  double z = c * u / (1.0 + std::sqrt(arg));
  double up = u;
  for (int j = 0; j < 5; ++j) {
    up *= u;
    z += a[j] * up;
  }
  return z;
}

// per-lens FP64 parameters not kept in the device image
struct HostExtra {
  double k[SD_MAX_SURFACES];
  double a[SD_MAX_SURFACES][5];
  double sd[SD_MAX_SURFACES];
};
HostExtra g_extra[SD_MAX_LENSES];

sd_status upload(const sd_lens* lens) {
  int dev = 0;
  SD_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != lens->device) return SD_ERR_ARG;
  SD_CUDA_TRY(cudaMemcpyToSymbol(c_lens, &lens->img, sizeof(DevLens),
                                 sizeof(DevLens) * lens->slot));
  return SD_OK;
}

void finish_image(DevLens& L, const HostExtra& X) {
  for (int s = 0; s < L.n; ++s) refresh_surface(L, s, &X.k[s], X.a[s], X.sd[s]);
  L.sd_stop = X.sd[L.stop];
  double zf = 0.0;
  if (L.type[0] == SD_SURF_REFRACT)
    zf = std::min(0.0, sag_at(L.c[0], X.k[0], X.a[0], X.sd[0]));
  L.z_front = zf;
}

}  // namespace
}  // namespace sd

extern "C" {

sd_status sd_lens_load(const sd_surface* surfs, int n, double focus_mm,
                       sd_lens** out) {
  SD_API_RANGE("sd_lens_load");
  using namespace sd;
  if (!surfs || !out || n < 1 || n > SD_MAX_SURFACES) return SD_ERR_ARG;
  if (!std::isfinite(focus_mm)) return SD_ERR_ARG;
  *out = nullptr;
  DevLens L;
  std::memset(&L, 0, sizeof L);
  HostExtra X;
  std::memset(&X, 0, sizeof X);
  L.n = n;
  L.stop = -1;
  for (int i = 0; i < n; ++i) {
    const sd_surface& s = surfs[i];
    if (s.type != SD_SURF_REFRACT && s.type != SD_SURF_STOP) return SD_ERR_LENS;
    double vals[] = {s.radius, s.thickness, s.nd, s.vd, s.semi_diameter, s.conic,
                     s.asph[0], s.asph[1], s.asph[2], s.asph[3], s.asph[4]};
    for (double v : vals)
      if (!fin(v)) return SD_ERR_LENS;
    if (s.nd < 1.0 || s.semi_diameter <= 0.0 || s.thickness < 0.0) return SD_ERR_LENS;
    if (s.type == SD_SURF_STOP) {
      if (L.stop >= 0) return SD_ERR_LENS;  // exactly one stop
      L.stop = i;
    }
    L.type[i] = s.type;
    L.c[i] = (s.type == SD_SURF_STOP || s.radius == 0.0) ? 0.0 : 1.0 / s.radius;
    L.t[i] = s.thickness;
    cauchy_fit(s.nd, s.vd, &L.A[i], &L.B[i]);
    X.k[i] = s.type == SD_SURF_STOP ? 0.0 : s.conic;
    for (int j = 0; j < 5; ++j) X.a[i][j] = s.type == SD_SURF_STOP ? 0.0 : s.asph[j];
    X.sd[i] = s.semi_diameter;
    if (s.type == SD_SURF_REFRACT &&
        1.0 - (1.0 + X.k[i]) * L.c[i] * L.c[i] * X.sd[i] * X.sd[i] < 0.0)
      return SD_ERR_LENS;  // aperture beyond the conic's rim
  }
  if (L.stop < 0) return SD_ERR_LENS;
  if (focus_mm > 0) {
    double nlam[SD_MAX_SURFACES];
    indices_at(L, 587.5618, nlam);
    double d = image_distance(L, nlam, focus_mm);
    if (!(d > 0) || !std::isfinite(d)) return SD_ERR_LENS;
    L.t[n - 1] = d;
  }
  if (!(L.t[n - 1] > 0)) return SD_ERR_LENS;
  finish_image(L, X);

  int dev = 0;
  SD_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  int slot = -1;
  for (int i = 0; i < SD_MAX_LENSES; ++i)
    if (!g_used[i]) {
      slot = i;
      break;
    }
  if (slot < 0) return SD_ERR_CAPACITY;
  sd_lens* lens = new sd_lens;
  lens->slot = slot;
  lens->device = dev;
  lens->img = L;
  g_extra[slot] = X;
  sd_status st = upload(lens);
  if (st != SD_OK) {
    delete lens;
    return st;
  }
  g_used[slot] = true;
  *out = lens;
  return SD_OK;
}

sd_status sd_lens_paraxial(const sd_lens* lens, double lambda_nm, double depth_mm,
                           sd_paraxial* out) {
  using namespace sd;
  if (!lens || !out || !(lambda_nm > 0) || !(depth_mm > 0)) return SD_ERR_ARG;
  const DevLens& L = lens->img;
  double nlam[SD_MAX_SURFACES];
  indices_at(L, lambda_nm, nlam);
  PYU r = parax(L, nlam, 1.0, 0.0, 0, L.n - 1);
  int s = L.n - 1;
  double n2 = nlam[s], u = r.u;
  if (L.type[s] == SD_SURF_REFRACT) u = (r.n * r.u - r.y * (n2 - r.n) * L.c[s]) / n2;
  out->efl = -1.0 / (n2 * u);
  out->bfl = -r.y / u;
  RayGen g = ray_gen(L, nlam, 1.0, depth_mm);
  out->z_ep = g.z_ep;
  out->r_ep = g.r_ep;
  out->sensor_dist = L.t[L.n - 1];
  out->m_sensor = 1.0 / g.x_o;
  out->img_dist = image_distance(L, nlam, depth_mm);
  double z = 0;
  for (int i = 0; i < L.n; ++i) z += L.t[i];
  out->z_sensor = z;
  return SD_OK;
}

sd_status sd_lens_set_param(sd_lens* lens, int pid, double value) {
  using namespace sd;
  if (!lens || !std::isfinite(value)) return SD_ERR_ARG;
  DevLens& L = lens->img;
  int s = pid / 8, j = pid % 8;
  if (pid < 0 || s >= L.n) return SD_ERR_ARG;
  HostExtra& X = g_extra[lens->slot];
  if (L.type[s] == SD_SURF_STOP && j != 7) return SD_ERR_ARG;
  if (j == 0)
    L.c[s] = value;
  else if (j == 1)
    X.k[s] = value;
  else if (j == 7) {
    if (value < 0 || (s == L.n - 1 && value <= 0)) return SD_ERR_LENS;
    L.t[s] = value;
  } else
    X.a[s][j - 2] = value;
  finish_image(L, X);
  return upload(lens);
}

sd_status sd_lens_free(sd_lens* lens) {
  if (!lens) return SD_ERR_ARG;
  std::lock_guard<std::mutex> lk(sd::g_mu);
  sd::g_used[lens->slot] = false;
  delete lens;
  return SD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Trace kernels
// ---------------------------------------------------------------------------
namespace sd {

enum { ST_OK = 0, ST_MISS = 1, ST_CLIP = 2, ST_TIR = 3, ST_NEWTON = 4, ST_BACK = 5,
       ST_NONE = 6 };  // ST_NONE: the empty slot of a pair past the last ray

struct SensorF {
  float ps, inv_ps, h, w, r2, fh;  // fh = (f - h) / f
  double ps_d;                     // pitch in FP64 (pixel positions of a map)
};

struct TraceParams {
  const sd_psf_request* req;
  int n_req;
  // per-pixel PSF map mode (req == nullptr): request r is pixel r of the
  // map_H x map_W depth map (metres), at its sensor position
  const float* map_depth;
  int map_H, map_W;
  double map_lambda_nm;
  int map_n, map_ks;
  int slots[SD_MAX_LENSES];
  int n_lenses;
  SensorF sen;
  int norm;
  int newton_max;
  int max_n;           // capacity of the row tables
  int max_ks;
  void* out;
  long long* stats;
  // landing mask (nullable): one bit per ray, mask_words words per request
  unsigned* land_mask;
  int mask_words;
  // hit dump (test path)
  float* rec;
  int max_rays;
  int* n_rays;
};

// Per-request context computed by the block prologue.
struct ReqCtx {
  float x_o, y_o;       // object point (x, y)
  float scale;          // pupil sample spacing r_ep / N
  float vz;             // z_ep + depth (axial length from p to the EP plane)
  float z_start, s_start, z_ep;
  float xc, yc;
  int slot, N, ks, total;
  int ok;
  float eta[SD_MAX_SURFACES];    // n_before / n_after at the request wavelength
  float omeg2[SD_MAX_SURFACES];  // 1 - eta^2 (evaluated in FP64)
};

// Integer square root floor(sqrt(v)) for 0 <= v < 2^24.
__device__ __forceinline__ int isqrt_floor(int v) {
  int r = (int)sqrtf((float)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

// Number of in-pupil samples of pupil row iy and the first column index.
__device__ __forceinline__ void row_span(int N, int iy, int* cnt, int* lo) {
  int b = 2 * iy + 1 - N;
  int rem = N * N - b * b;
  int am = isqrt_floor(rem);
  // a = 2 ix + 1 - N has the parity of N + 1: largest such |a| <= sqrt(rem)
  if ((am + N + 1) & 1) am -= 1;
  *cnt = am + 1;
  *lo = (N - 1 - am) >> 1;
}

// Request r of the launch: from the request array, or in map mode built
// for pixel r of the depth map (image position of the pixel centre relative
// to the sensor centre, the pixel's depth, PSF at offset r * 2 ks^2).
__device__ __forceinline__ sd_psf_request request_of(const TraceParams& P, int r) {
  if (!P.map_depth) return P.req[r];
  sd_psf_request q;
  const int row = r / P.map_W, col = r - row * P.map_W;
  const double ps = (double)P.sen.ps_d;
  q.h_mm = ((double)col - 0.5 * (double)(P.map_W - 1)) * ps;
  q.v_mm = ((double)row - 0.5 * (double)(P.map_H - 1)) * ps;
  q.depth_mm = (double)P.map_depth[r] * 1000.0;
  q.lambda_nm = P.map_lambda_nm;
  q.n_grid = P.map_n;
  q.ks = P.map_ks;
  q.lens = 0;
  q.reserved = 0;
  q.out_offset = (long long)r * 2 * P.map_ks * P.map_ks;
  return q;
}

// Block prologue: paraxial set-up (FP64, thread 0) and pupil row tables.
__device__ void setup_request(const TraceParams& P, const sd_psf_request& q,
                              ReqCtx& ctx, int* prefix, int* lo) {
  if (threadIdx.x == 0) {
    int li = q.lens;
    ctx.ok = (li >= 0 && li < P.n_lenses && q.n_grid >= 2 && q.n_grid <= P.max_n &&
              q.ks >= 1 && (q.ks & 1) && q.ks <= P.max_ks && q.depth_mm > 0 &&
              q.lambda_nm > 0);
    if (ctx.ok) {
      int slot = P.slots[li];
      const DevLens& L = c_lens[slot];
      double nlam[SD_MAX_SURFACES];
      indices_at(L, q.lambda_nm, nlam);
      double nb = 1.0;
      for (int s = 0; s < L.n; ++s) {
        double e = nb / nlam[s];
        ctx.eta[s] = (float)e;
        ctx.omeg2[s] = (float)(1.0 - e * e);
        nb = nlam[s];
      }
      RayGen g = ray_gen(L, nlam, q.h_mm, q.depth_mm);
      ctx.x_o = (float)g.x_o;
      ctx.y_o = (float)(q.v_mm / g.m);
      ctx.scale = (float)(g.r_ep / q.n_grid);
      ctx.vz = (float)(g.z_ep + q.depth_mm);
      ctx.z_ep = (float)g.z_ep;
      ctx.z_start = (float)g.z_start;
      ctx.s_start = (float)((g.z_start + q.depth_mm) / (g.z_ep + q.depth_mm));
      ctx.xc = (float)q.h_mm;
      ctx.yc = (float)q.v_mm;
      ctx.slot = slot;
      ctx.N = q.n_grid;
      ctx.ks = q.ks;
    } else {
      ctx.N = 0;
      ctx.ks = 0;
    }
  }
  __syncthreads();
  int N = ctx.N;
  // pupil row spans, then an exclusive prefix over rows (one warp scans)
  for (int iy = threadIdx.x; iy < N; iy += blockDim.x) {
    int c, l;
    row_span(N, iy, &c, &l);
    prefix[iy + 1] = c;
    lo[iy] = l;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    int lane = threadIdx.x;
    int carry = 0;
    for (int base = 0; base < N; base += 32) {
      int i = base + lane;
      int v = (i < N) ? prefix[i + 1] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      if (i < N) prefix[i + 1] = v + carry;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) {
      prefix[0] = 0;
      ctx.total = carry;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// One ray (float) or two rays (float2) through the same rounded operations.
// The tracer below is written once over these: every FP32 operation is an
// explicitly rounded add, multiply or fused multiply-add (no contraction left
// to the compiler), and the float2 forms are the packed two-lane
// instructions of sm_100 and later, whose components round exactly like the
// scalar ones.  So a ray traced alone and the same ray traced as one of a
// pair give the same bits, and the forward (pairs), the adjoint's recompute,
// the batched trace and the map trace (single rays) take the same decisions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
// a - b = a + (-b) with one rounding
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, vneg(b)); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <class V> __device__ __forceinline__ V vb(float s);
template <> __device__ __forceinline__ float vb<float>(float s) { return s; }
template <> __device__ __forceinline__ float2 vb<float2>(float s) { return make_float2(s, s); }

// Hardware reciprocal estimate (rcp.approx, about 1 ulp; denormals flushed).
__device__ __forceinline__ float rcp_est(float b) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(b));
  return r;
}
__device__ __forceinline__ float2 rcp_est(float2 b) { return make_float2(rcp_est(b.x), rcp_est(b.y)); }
__device__ __forceinline__ float rsqrt_est(float x) { return rsqrtf(x); }
__device__ __forceinline__ float2 rsqrt_est(float2 x) { return make_float2(rsqrtf(x.x), rsqrtf(x.y)); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float2 vmax(float2 a, float b) {
  return make_float2(fmaxf(a.x, b), fmaxf(a.y, b));
}
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float2 fast_div(float2 a, float2 b) {
  return make_float2(__fdividef(a.x, b.x), __fdividef(a.y, b.y));
}

// Per-ray masks and statuses: bool / int for one ray, two of each for a pair.
struct M2 {
  bool x, y;
};
__device__ __forceinline__ bool lt(float a, float b) { return a < b; }
__device__ __forceinline__ M2 lt(float2 a, float b) { return {a.x < b, a.y < b}; }
__device__ __forceinline__ bool gt(float a, float b) { return a > b; }
__device__ __forceinline__ M2 gt(float2 a, float b) { return {a.x > b, a.y > b}; }
__device__ __forceinline__ M2 gt(float2 a, float2 b) { return {a.x > b.x, a.y > b.y}; }
__device__ __forceinline__ bool vnot(bool m) { return !m; }
__device__ __forceinline__ M2 vnot(M2 m) { return {!m.x, !m.y}; }
__device__ __forceinline__ bool vand(bool a, bool b) { return a && b; }
__device__ __forceinline__ M2 vand(M2 a, M2 b) { return {a.x && b.x, a.y && b.y}; }
__device__ __forceinline__ bool any_of(bool m) { return m; }
__device__ __forceinline__ bool any_of(M2 m) { return m.x || m.y; }
__device__ __forceinline__ float sel(bool m, float a, float b) { return m ? a : b; }
__device__ __forceinline__ float2 sel(M2 m, float2 a, float2 b) {
  return make_float2(m.x ? a.x : b.x, m.y ? a.y : b.y);
}
__device__ __forceinline__ bool small_step(float s) { return fabsf(s) < 1e-5f; }
__device__ __forceinline__ M2 small_step(float2 s) { return {fabsf(s.x) < 1e-5f, fabsf(s.y) < 1e-5f}; }

// status: the first failure of each ray stays
__device__ __forceinline__ int fail(int st, bool m, int code) { return st == ST_OK && m ? code : st; }
__device__ __forceinline__ int2 fail(int2 st, M2 m, int code) {
  return make_int2(st.x == ST_OK && m.x ? code : st.x, st.y == ST_OK && m.y ? code : st.y);
}
__device__ __forceinline__ bool dead(int st) { return st != ST_OK; }
__device__ __forceinline__ bool dead(int2 st) { return st.x != ST_OK && st.y != ST_OK; }
__device__ __forceinline__ bool alive(int st) { return st == ST_OK; }
__device__ __forceinline__ M2 alive(int2 st) { return {st.x == ST_OK, st.y == ST_OK}; }
template <class V> struct VStat;
template <> struct VStat<float> {
  using S = int;
  using M = bool;
};
template <> struct VStat<float2> {
  using S = int2;
  using M = M2;
};

// a*b + c*d with one rounding to about 1 ulp (Kahan: the rounding error of
// c*d is recovered exactly by an FMA and added back)
template <class V>
__device__ __forceinline__ V dot2(V a, V b, V c, V d) {
  const V w = vmul(c, d);
  const V e = vfma(c, d, vneg(w));
  const V f = vfma(a, b, w);
  return vadd(f, e);
}

// 1/sqrt(x) to about half an ulp: hardware estimate plus one Newton step
// (unit vectors feed Snell's law, whose output direction error is
// multiplied by the remaining path length to the sensor).
template <class V>
__device__ __forceinline__ V rsqrt_refined(V x) {
  const V r = rsqrt_est(x);
  return vmul(r, vfma(vmul(vmul(vb<V>(-0.5f), x), r), r, vb<V>(1.5f)));
}

// a / b from the reciprocal estimate and one Newton-Raphson correction of
// the quotient (Markstein, IBM J. Res. Dev. 34(1), 1990): the FMA residual
// a - b q0 of q0 = a rcp(b) is exact, and q0 + residual * rcp(b) is within
// one ulp of a / b.  Branch-free; valid for the normal-range operands of the
// trace (lengths and cosines), b != 0.
template <class V>
__device__ __forceinline__ V div_nr(V a, V b) {
  const V r = rcp_est(b);
  const V q = vmul(a, r);
  return vfma(vfma(vneg(b), q, a), r, q);
}

// sqrt(x) for x >= 0 from the reciprocal square-root estimate and one
// Newton correction on the residual x - s^2 (Markstein's method), within
// about one ulp.  x is clamped to 1e-30 so that x = 0 yields 1e-15, not NaN.
template <class V>
__device__ __forceinline__ V sqrt_nr(V x) {
  x = vmax(x, 1e-30f);
  const V r = rsqrt_est(x);
  const V s = vmul(x, r);
  return vfma(vfma(vneg(s), s, x), vmul(vb<V>(0.5f), r), s);
}

// Constants of surface s for the tracer, derived with explicitly rounded
// operations from the lens image and the request's refractive ratios: as
// values (one ray) or as duplicated pairs (two rays) staged per block.
template <class V>
struct SurfK {
  V c, negc, k, kk;    // curvature, its negative, conic, 1 + k
  V nkc2, halfc;       // -(1 + k) c^2, c / 2
  V negckk, sd2, negt; // -c (1 + k), clear semi-diameter^2, -thickness
  V a[5], da[5];       // a4..a12 and m a_2m
  V e, e2, om;         // eta, eta^2, 1 - eta^2
  // for the adjoint's reverse sweep
  V ie, ie2;           // 1 / eta, its square
  V kc2, qc3, qkc3;    // (1 + k) c^2, c^3 / 4, (1 + k) c^3 / 4
  V dda[5];            // (m - 1) m a_2m
  int kind;
};

__device__ __forceinline__ SurfK<float> surf_consts(const DevSurf& S, float eta, float omeg2) {
  SurfK<float> K;
  K.c = S.c;
  K.negc = -S.c;
  K.k = S.k;
  K.kk = __fadd_rn(1.f, S.k);
  K.nkc2 = -__fmul_rn(__fmul_rn(K.kk, S.c), S.c);
  K.halfc = __fmul_rn(0.5f, S.c);
  K.negckk = -__fmul_rn(S.c, K.kk);
  K.sd2 = S.sd2;
  K.negt = -S.t;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    K.a[j] = S.a[j];
    K.da[j] = S.da[j];
  }
  K.e = eta;
  K.e2 = __fmul_rn(eta, eta);
  K.om = omeg2;
  K.ie = div_nr(1.f, eta);
  K.ie2 = __fmul_rn(K.ie, K.ie);
  K.kc2 = __fmul_rn(__fmul_rn(K.kk, S.c), S.c);
  K.qc3 = __fmul_rn(0.25f, __fmul_rn(__fmul_rn(S.c, S.c), S.c));
  K.qkc3 = __fmul_rn(K.kk, K.qc3);
#pragma unroll
  for (int j = 0; j < 5; ++j) K.dda[j] = __fmul_rn((float)(j + 1), S.da[j]);
  K.kind = S.kind;
  return K;
}

__device__ __forceinline__ SurfK<float2> pair_consts(const SurfK<float>& K) {
  SurfK<float2> P;
  P.c = vb<float2>(K.c);
  P.negc = vb<float2>(K.negc);
  P.k = vb<float2>(K.k);
  P.kk = vb<float2>(K.kk);
  P.nkc2 = vb<float2>(K.nkc2);
  P.halfc = vb<float2>(K.halfc);
  P.negckk = vb<float2>(K.negckk);
  P.sd2 = vb<float2>(K.sd2);
  P.negt = vb<float2>(K.negt);
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    P.a[j] = vb<float2>(K.a[j]);
    P.da[j] = vb<float2>(K.da[j]);
  }
  P.e = vb<float2>(K.e);
  P.e2 = vb<float2>(K.e2);
  P.om = vb<float2>(K.om);
  P.ie = vb<float2>(K.ie);
  P.ie2 = vb<float2>(K.ie2);
  P.kc2 = vb<float2>(K.kc2);
  P.qc3 = vb<float2>(K.qc3);
  P.qkc3 = vb<float2>(K.qkc3);
#pragma unroll
  for (int j = 0; j < 5; ++j) P.dda[j] = vb<float2>(K.dda[j]);
  P.kind = K.kind;
  return P;
}

// Sequential trace (FP32) of one ray (V = float) or two rays (V = float2)
// in surface-0-vertex-local coordinates; KS(s) yields SurfK<V> of surface s.
// On success (x, y) is the sensor landing point and (dx, dy, dz) the unit
// direction.  Positions are kept relative to the current surface vertex.
// A ray of a pair that fails keeps its first status and runs on with the
// other (its values are not used); loops end when both rays are done.
// Per-surface forward state kept for the adjoint (SAVE): the intersection
// parameter at every surface and the last hit point, of one ray or a pair.
template <class V>
struct AdjStateV {
  V t[SD_MAX_SURFACES];  // intersection parameter at every surface
  V px, py, pz;          // hit point at the last surface (vertex-local)
};
using AdjState = AdjStateV<float>;

// A single ray returns at its first failure; a pair runs each surface to its
// end and returns there when both rays have failed (fewer tests per ray).
#define SD_EARLY_OUT(V, st)                          \
  if constexpr (std::is_same<V, float>::value) {     \
    if (dead(st)) return st;                         \
  }

template <bool SAVE, class V, class KS>
__device__ __forceinline__ typename VStat<V>::S trace_ray_v(
    int n, const KS& ks_of, int newton_max, typename VStat<V>::S st, V& x, V& y, V& z, V& dx,
    V& dy, V& dz, AdjStateV<V>* sv) {
  using M = typename VStat<V>::M;
  const V one = vb<V>(1.f), m2 = vb<V>(-2.f);
  for (int s = 0; s < n; ++s) {
    const SurfK<V>& S = ks_of(s);
    const int kind = S.kind;
    V t;
    if (kind & K_FLAT) {
      st = fail(st, vnot(gt(dz, 0.f)), ST_BACK);
      SD_EARLY_OUT(V, st);
      t = div_nr(vneg(z), dz);
    } else {
      // conic: A t^2 - 2 B t + C = 0 (|d| = 1), root nearest the vertex in
      // the cancellation-free form t = C / (B + sqrt(B^2 - A C)); nA = -A
      const V nA = vmul(S.negc, vfma(vmul(S.k, dz), dz, one));
      const V kz = vmul(S.kk, z);
      const V B = vfma(S.negc, vfma(kz, dz, vfma(y, dy, vmul(x, dx))), dz);
      const V C = vfma(S.c, vfma(kz, z, vfma(y, y, vmul(x, x))), vmul(m2, z));
      const V disc = vfma(nA, C, vmul(B, B));
      const V den = vadd(B, sqrt_nr(disc));
      // no real root, or the root's denominator not positive
      st = fail(st, vnot(vand(vnot(lt(disc, 0.f)), gt(den, 0.f))), ST_MISS);
      SD_EARLY_OUT(V, st);
      t = div_nr(C, den);
    }
    if (kind & K_ASPH) {
      // Newton on F(t) = z + t dz - sag(rho(t)^2), started at the conic root;
      // a ray stops updating t once its step is below 1e-5 mm
      M act = alive(st);
      int it = 0;
      for (; it < newton_max; ++it) {
        const V px = vfma(t, dx, x), py = vfma(t, dy, y);
        const V u = vfma(py, py, vmul(px, px));
        const V arg = vfma(S.nkc2, u, one);
        st = fail(st, vand(act, lt(arg, 0.f)), ST_NEWTON);
        act = vand(act, alive(st));
        if (!any_of(act)) break;
        const V argc = vmax(arg, 1e-30f);
        const V r = rsqrt_est(argc);
        // q = sqrt(arg) (sqrt_nr, sharing the estimate with the derivative)
        const V s0 = vmul(argc, r);
        const V q = vfma(vfma(vneg(s0), s0, argc), vmul(vb<V>(0.5f), r), s0);
        const V poly =
            vfma(u, vfma(u, vfma(u, vfma(u, S.a[4], S.a[3]), S.a[2]), S.a[1]), S.a[0]);
        const V zs = vfma(vmul(u, u), poly, div_nr(vmul(S.c, u), vadd(one, q)));
        const V dpoly =
            vfma(u, vfma(u, vfma(u, vfma(u, S.da[4], S.da[3]), S.da[2]), S.da[1]), S.da[0]);
        // the derivative and the step only steer the iteration (its fixed
        // point is the root of the exactly evaluated F): estimates suffice
        const V dzdu = vfma(u, dpoly, vmul(S.halfc, r));
        const V F = vsub(vfma(t, dz, z), zs);
        const V dF = vfma(vmul(m2, dzdu), vfma(py, dy, vmul(px, dx)), dz);
        const V step = fast_div(F, dF);
        t = vsub(t, sel(act, step, vb<V>(0.f)));
        act = vand(act, vnot(small_step(step)));
        if (!any_of(act)) break;
      }
      st = fail(st, act, ST_NEWTON);  // not converged in newton_max steps
      SD_EARLY_OUT(V, st);
    }
    if constexpr (SAVE) sv->t[s] = t;
    x = vfma(t, dx, x);
    y = vfma(t, dy, y);
    z = vfma(t, dz, z);
    if constexpr (SAVE) {
      if (s == n - 1) {
        sv->px = x;
        sv->py = y;
        sv->pz = z;
      }
    }
    const V rho2 = vfma(y, y, vmul(x, x));
    st = fail(st, gt(rho2, S.sd2), ST_CLIP);
    SD_EARLY_OUT(V, st);
    if (kind & K_REFRACT) {
      V nx, ny, nz;
      if (kind & K_ASPH) {
        const V qq = sqrt_nr(vfma(S.nkc2, rho2, one));
        const V dpoly = vfma(
            rho2, vfma(rho2, vfma(rho2, vfma(rho2, S.da[4], S.da[3]), S.da[2]), S.da[1]),
            S.da[0]);
        const V dzdu = vfma(rho2, dpoly, div_nr(S.halfc, qq));
        nx = vmul(vmul(m2, x), dzdu);
        ny = vmul(vmul(m2, y), dzdu);
        nz = one;
      } else {
        // gradient of the quadric c(x^2+y^2) + c(1+k) z^2 - 2 z, oriented +z
        nx = vmul(S.negc, x);
        ny = vmul(S.negc, y);
        nz = vfma(S.negckk, z, one);
      }
      const V inv = rsqrt_refined(vfma(nz, nz, vfma(ny, ny, vmul(nx, nx))));
      nx = vmul(nx, inv);
      ny = vmul(ny, inv);
      nz = vmul(nz, inv);
      // vector Snell's law with the normal along the propagation:
      // d' = e d + g n with g = cos(t_t) - e cos(t_i), evaluated as
      // (1 - e^2) / (cos(t_t) + e cos(t_i)) to avoid the cancellation;
      // cos^2(t_t) = 1 - e^2 (1 - cos^2(t_i)) = (1 - e^2) + e^2 cos^2(t_i)
      const V cosi = vfma(nz, dz, vfma(ny, dy, vmul(nx, dx)));
      const V k2 = vfma(vmul(S.e2, cosi), cosi, S.om);
      st = fail(st, lt(k2, 0.f), ST_TIR);
      SD_EARLY_OUT(V, st);
      const V g = div_nr(S.om, vfma(S.e, cosi, sqrt_nr(k2)));
      dx = dot2(S.e, dx, g, nx);
      dy = dot2(S.e, dy, g, ny);
      dz = dot2(S.e, dz, g, nz);
    }
    z = vadd(z, S.negt);  // vertex-local coordinate of the next surface (or the sensor)
    if (dead(st)) return st;
  }
  st = fail(st, vnot(gt(dz, 0.f)), ST_BACK);
  if (dead(st)) return st;
  const V t = div_nr(vneg(z), dz);
  x = vfma(t, dx, x);
  y = vfma(t, dy, y);
  return st;
}

// One ray, the surface constants derived on the fly (the adjoint, the
// batched trace, the map trace, the hit dump).
template <bool SAVE>
__device__ __forceinline__ int trace_ray_t(int slot, const float* __restrict__ eta,
                                           const float* __restrict__ omeg2, int newton_max,
                                           float& x, float& y, float& z, float& dx, float& dy,
                                           float& dz, AdjState* sv) {
  const DevLens& L = c_lens[slot];
  auto ks_of = [&](int s) { return surf_consts(L.s[s], eta[s], omeg2[s]); };
  return trace_ray_v<SAVE, float>(L.n, ks_of, newton_max, (int)ST_OK, x, y, z, dx, dy, dz, sv);
}

__device__ __forceinline__ int trace_ray(int slot, const float* __restrict__ eta,
                                         const float* __restrict__ omeg2, int newton_max,
                                         float& x, float& y, float& z,
                                         float& dx, float& dy, float& dz) {
  return trace_ray_t<false>(slot, eta, omeg2, newton_max, x, y, z, dx, dy, dz, nullptr);
}

// tan(theta) = D_x / D_z of a landing ray (Sec. 3.1).  It enters the decision
// only through h tan(theta) with h ~ 1e-3 mm, so a 2-ulp quotient is ample;
// every path (forward, hit dump, adjoint) uses this one expression.
__device__ __forceinline__ float tan_theta(float dx, float dz) { return __fdividef(dx, dz); }

// Eq. (1)/(2): s = offset on the sub-pixel plane relative to the pixel centre;
// L for 0 <= s < w, R for -w <= s < 0, else missed.
__device__ __forceinline__ int dp_side(const SensorF& S, float dxp, float dyp, float tan_t) {
  bool inside = dxp * dxp + dyp * dyp <= S.r2;
  float s = inside ? fmaf(dxp, S.fh, S.h * tan_t) : fmaf(S.h, tan_t, dxp);
  if (s >= 0.f && s < S.w) return 0;
  if (s >= -S.w && s < 0.f) return 1;
  return 2;
}

// Generates ray k of the request (in pupil raster order over in-pupil samples).
// Ray through pupil sample (ix, iy) of the request: from the object point
// to the sample on the EP plane, started on that plane (or on the start
// plane in front of surface 0).
__device__ __forceinline__ void pupil_ray(const ReqCtx& ctx, int ix, int iy, float& x, float& y,
                                          float& z, float& dx, float& dy, float& dz) {
  const int N = ctx.N;
  float ex = (float)(2 * ix + 1 - N) * ctx.scale;
  float ey = (float)(2 * iy + 1 - N) * ctx.scale;
  float vx = ex - ctx.x_o, vy = ey - ctx.y_o, vz = ctx.vz;
  float inv = rsqrt_refined(vx * vx + vy * vy + vz * vz);
  dx = vx * inv;
  dy = vy * inv;
  dz = vz * inv;
  if (ctx.s_start == 1.f) {
    x = ex;
    y = ey;
  } else {
    x = fmaf(ctx.s_start, vx, ctx.x_o);
    y = fmaf(ctx.s_start, vy, ctx.y_o);
  }
  z = ctx.z_start;
}

// Ray k given its pupil row iy (prefix[iy] <= k < prefix[iy+1]).
__device__ __forceinline__ void make_ray_row(const ReqCtx& ctx, const int* prefix, const int* lo,
                                             int k, int iy, float& x, float& y, float& z,
                                             float& dx, float& dy, float& dz) {
  pupil_ray(ctx, lo[iy] + (k - prefix[iy]), iy, x, y, z, dx, dy, dz);
}

// Ray k of the request (binary search for its pupil row).
__device__ __forceinline__ void make_ray(const ReqCtx& ctx, const int* prefix, const int* lo,
                                         int k, float& x, float& y, float& z, float& dx,
                                         float& dy, float& dz) {
  int a = 0, b = ctx.N;
  while (b - a > 1) {
    int m = (a + b) >> 1;
    if (prefix[m] <= k) a = m; else b = m;
  }
  make_ray_row(ctx, prefix, lo, k, a, x, y, z, dx, dy, dz);
}

// Pupil row of ray k for a thread whose k only grows: advance from the row
// of its previous ray (a few steps instead of a binary search).
__device__ __forceinline__ int advance_row(const int* prefix, int k, int row) {
  while (prefix[row + 1] <= k) ++row;
  return row;
}

// bytes of the pupil row tables (prefix[N+1], lo[N]), 16-byte multiple
__host__ __device__ inline size_t table_bytes(int max_n) {
  return (((size_t)(2 * max_n + 1) * 4) + 15) & ~(size_t)15;
}

template <class OutT>
__device__ __forceinline__ void store_out(void* out, long long idx, float v) {
  reinterpret_cast<OutT*>(out)[idx] = from_f32<OutT>(v);
}

// One block per request.  MODE 0: hard counts (u32), 1: bilinear (f32).
// A thread traces rays k and k + blockDim.x together (packed pairs) and bins
// each of the two sets of blockDim.x consecutive rays as one.
template <int MODE, class OutT>
__global__ void __launch_bounds__(256) trace_bin_kernel(TraceParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ReqCtx ctx;
  __shared__ SurfK<float2> s_surf[SD_MAX_SURFACES];
  __shared__ unsigned int s_stats[SD_N_STATS];
  __shared__ float s_red[2][32];
  int* prefix = reinterpret_cast<int*>(smem);
  int* lo = prefix + (P.max_n + 1);
  unsigned int* patch = reinterpret_cast<unsigned int*>(smem + table_bytes(P.max_n));
  float* patchf = reinterpret_cast<float*>(patch);

  const int r = blockIdx.x;
  const sd_psf_request q = request_of(P, r);
  if (threadIdx.x < SD_N_STATS) s_stats[threadIdx.x] = 0;
  setup_request(P, q, ctx, prefix, lo);
  const int ks = ctx.ks, ks2 = ks * ks, p = (ks - 1) >> 1;
  for (int i = threadIdx.x; i < 2 * ks2; i += blockDim.x) patch[i] = 0u;
  const int nsurf = ctx.N ? c_lens[ctx.slot].n : 0;
  for (int sf = threadIdx.x; sf < nsurf; sf += blockDim.x)
    s_surf[sf] = pair_consts(surf_consts(c_lens[ctx.slot].s[sf], ctx.eta[sf], ctx.omeg2[sf]));
  __syncthreads();

  const SensorF S = P.sen;
  const int total = ctx.N ? ctx.total : 0;
  const int lane = threadIdx.x & 31;
  unsigned int c_reached = 0, c_vign = 0, c_other = 0, c_l = 0, c_r = 0, c_miss = 0,
               c_clip = 0;
  auto ks_of = [&](int sf) -> const SurfK<float2>& { return s_surf[sf]; };
  // bins one ray (k, its status and landing values) of a set of blockDim.x
  // consecutive rays; every thread of the block calls it for each set
  auto bin = [&](int k, int st, float x, float y, float dx, float dz) {
    int key = -1;
    float fx = 0.f, fy = 0.f;
    int side = 2;
    // lands on the L or R sub-pixel with its nearest pixel centre at most one
    // pixel outside the patch (the adjoint takes the same decisions)
    bool land = false;
    if (k < total) {
      if (st == ST_OK) {
        ++c_reached;
        fx = (x - ctx.xc) * S.inv_ps + (float)p;
        fy = (y - ctx.yc) * S.inv_ps + (float)p;
        float af = floorf(fx + 0.5f), bf = floorf(fy + 0.5f);
        side = dp_side(S, (fx - af) * S.ps, (fy - bf) * S.ps, tan_theta(dx, dz));
        bool inpatch = af >= 0.f && af < (float)ks && bf >= 0.f && bf < (float)ks;
        land = side != 2 && af >= -1.f && af <= (float)ks && bf >= -1.f && bf <= (float)ks;
        if (!inpatch) {
          ++c_clip;
          if (MODE == 0) side = 2;  // nothing to deposit
        } else if (side == 2) {
          ++c_miss;
        } else {
          if (side == 0) ++c_l; else ++c_r;
        }
        if (MODE == 0 && inpatch && side < 2) key = side * ks2 + (int)bf * ks + (int)af;
      } else if (st == ST_CLIP) {
        ++c_vign;
      } else {
        ++c_other;
      }
    }
    if (P.land_mask) {
      // one word per warp: its 32 consecutive rays k - lane .. k - lane + 31
      const unsigned bits = __ballot_sync(0xffffffffu, land);
      const int kw = k - lane;
      if (lane == 0 && kw < total && SD_CHECK(kw >> 5, P.mask_words))
        P.land_mask[(size_t)r * P.mask_words + (kw >> 5)] = bits;
    }
    if (MODE == 0) {
      // warp-aggregated shared-memory increment of the landing bin
      unsigned int m = __match_any_sync(0xffffffffu, key);
      if (key >= 0 && lane == __ffs(m) - 1 && SD_CHECK(key, 2 * ks2))
        atomicAdd(&patch[key], (unsigned)__popc(m));
    } else if (side < 2) {
      float a0f = floorf(fx), b0f = floorf(fy);
      float wx = fx - a0f, wy = fy - b0f;
      int a0 = (int)a0f, b0 = (int)b0f;
      float* P0 = patchf + side * ks2;
#pragma unroll
      for (int jy = 0; jy < 2; ++jy)
#pragma unroll
        for (int jx = 0; jx < 2; ++jx) {
          int aa = a0 + jx, bb = b0 + jy;
          if (aa >= 0 && aa < ks && bb >= 0 && bb < ks)
            atomicAdd(&P0[bb * ks + aa], (jx ? wx : 1.f - wx) * (jy ? wy : 1.f - wy));
        }
    }
  };
  const int NT = blockDim.x;
  int row0 = 0, row1 = 0;
  for (int base = 0; base < total; base += 2 * NT) {
    const int k0 = base + threadIdx.x, k1 = k0 + NT;
    float2 x = make_float2(0.f, 0.f), y = x, z = x, dx = x, dy = x,
           dz = make_float2(1.f, 1.f);
    int2 st = make_int2(k0 < total ? (int)ST_OK : (int)ST_NONE,
                        k1 < total ? (int)ST_OK : (int)ST_NONE);
    if (k0 < total) {
      row0 = advance_row(prefix, k0, row0);
      make_ray_row(ctx, prefix, lo, k0, row0, x.x, y.x, z.x, dx.x, dy.x, dz.x);
    }
    if (k1 < total) {
      row1 = advance_row(prefix, k1, row1);
      make_ray_row(ctx, prefix, lo, k1, row1, x.y, y.y, z.y, dx.y, dy.y, dz.y);
    }
    if (k0 < total)
      st = trace_ray_v<false, float2>(nsurf, ks_of, P.newton_max, st, x, y, z, dx, dy, dz,
                                      nullptr);
    bin(k0, st.x, x.x, y.x, dx.x, dz.x);
    bin(k1, st.y, x.y, y.y, dx.y, dz.y);
  }
  // block statistics
  atomicAdd(&s_stats[SD_STAT_REACHED], c_reached);
  atomicAdd(&s_stats[SD_STAT_VIGNETTED], c_vign);
  atomicAdd(&s_stats[SD_STAT_OTHER], c_other);
  atomicAdd(&s_stats[SD_STAT_L], c_l);
  atomicAdd(&s_stats[SD_STAT_R], c_r);
  atomicAdd(&s_stats[SD_STAT_DP_MISSED], c_miss);
  atomicAdd(&s_stats[SD_STAT_CLIPPED], c_clip);
  __syncthreads();

  // sums of the L and R planes for the normalisation
  float sl = 0.f, sr = 0.f;
  for (int i = threadIdx.x; i < ks2; i += blockDim.x) {
    if (MODE == 0) {
      sl += (float)patch[i];
      sr += (float)patch[ks2 + i];
    } else {
      sl += patchf[i];
      sr += patchf[ks2 + i];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sl += __shfl_xor_sync(0xffffffffu, sl, o);
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
  }
  if (lane == 0) {
    s_red[0][threadIdx.x >> 5] = sl;
    s_red[1][threadIdx.x >> 5] = sr;
  }
  __syncthreads();
  float SL = 0.f, SR = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    SL += s_red[0][w];
    SR += s_red[1][w];
  }
  float scl = 1.f, scr = 1.f;
  if (P.norm == SD_NORM_JOINT) {
    float s = SL + SR;
    scl = scr = s > 0.f ? 1.f / s : 0.f;
  } else if (P.norm == SD_NORM_SEPARATE) {
    scl = SL > 0.f ? 1.f / SL : 0.f;
    scr = SR > 0.f ? 1.f / SR : 0.f;
  } else if (P.norm == SD_NORM_PER_RAY) {
    scl = scr = total > 0 ? 1.f / (float)total : 0.f;
  }
  if (ctx.N) {
    long long base = q.out_offset;
    for (int i = threadIdx.x; i < 2 * ks2; i += blockDim.x) {
      float v = (MODE == 0) ? (float)patch[i] : patchf[i];
      store_out<OutT>(P.out, base + i, v * (i < ks2 ? scl : scr));
    }
  }
  if (P.stats && threadIdx.x < SD_N_STATS) {
    long long v = threadIdx.x == SD_STAT_LAUNCHED ? (long long)total
                                                   : (long long)s_stats[threadIdx.x];
    P.stats[(long long)r * SD_N_STATS + threadIdx.x] = v;
  }
}

// Per-ray records of one request (test path).
__global__ void __launch_bounds__(256) trace_hits_kernel(TraceParams P, sd_psf_request q) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ReqCtx ctx;
  int* prefix = reinterpret_cast<int*>(smem);
  int* lo = prefix + (P.max_n + 1);
  setup_request(P, q, ctx, prefix, lo);
  const SensorF S = P.sen;
  const int ks = ctx.ks, p = (ks - 1) >> 1;
  const int total = ctx.N ? ctx.total : 0;
  if (threadIdx.x == 0) *P.n_rays = total;
  for (int k = threadIdx.x; k < total && k < P.max_rays; k += blockDim.x) {
    float x, y, z, dx, dy, dz;
    make_ray(ctx, prefix, lo, k, x, y, z, dx, dy, dz);
    int st = trace_ray(ctx.slot, ctx.eta, ctx.omeg2, P.newton_max, x, y, z, dx, dy, dz);
    float* o = P.rec + (long long)k * 8;
    float side = 2.f, pix = -1.f;
    if (st == ST_OK) {
      float fx = (x - ctx.xc) * S.inv_ps + (float)p;
      float fy = (y - ctx.yc) * S.inv_ps + (float)p;
      float af = floorf(fx + 0.5f), bf = floorf(fy + 0.5f);
      side = (float)dp_side(S, (fx - af) * S.ps, (fy - bf) * S.ps, tan_theta(dx, dz));
      if (af >= 0.f && af < (float)ks && bf >= 0.f && bf < (float)ks) pix = bf * 65536.f + af;
    } else {
      x = y = dx = dy = dz = 0.f;
    }
    o[0] = x;
    o[1] = y;
    o[2] = dx;
    o[3] = dy;
    o[4] = dz;
    o[5] = (float)st;
    o[6] = side;
    o[7] = pix;
  }
}

size_t trace_smem_bytes(int max_n, int max_ks) {
  return table_bytes(max_n) + (size_t)2 * max_ks * max_ks * 4;
}

__global__ void math_check_kernel(const float* a, const float* b, int n, float* quot,
                                  float* root) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    quot[i] = div_nr(a[i], b[i]);
    root[i] = sqrt_nr(a[i]);
  }
}

sd_status fill_params(TraceParams& P, const sd_lens* const* lenses, int n_lenses,
                      const sd_dp_sensor* sensor, const sd_trace_opts* opts) {
  if (!lenses || n_lenses < 1 || n_lenses > SD_MAX_LENSES || !sensor) return SD_ERR_ARG;
  int dev = 0;
  SD_CUDA_TRY(cudaGetDevice(&dev));
  for (int i = 0; i < n_lenses; ++i) {
    if (!lenses[i] || lenses[i]->device != dev) return SD_ERR_ARG;
    P.slots[i] = lenses[i]->slot;
  }
  P.n_lenses = n_lenses;
  const sd_dp_sensor& s = *sensor;
  if (!(s.pitch_mm > 0) || !(s.f_mm > s.h_mm) || s.h_mm < 0 || !(s.w_mm > 0) ||
      s.r_mm < 0)
    return SD_ERR_ARG;
  P.sen.ps = (float)s.pitch_mm;
  P.sen.ps_d = s.pitch_mm;
  P.sen.inv_ps = (float)(1.0 / s.pitch_mm);
  P.sen.h = (float)s.h_mm;
  P.sen.w = (float)s.w_mm;
  P.sen.r2 = (float)(s.r_mm * s.r_mm);
  P.sen.fh = (float)((s.f_mm - s.h_mm) / s.f_mm);
  P.norm = opts ? opts->norm : SD_NORM_JOINT;
  if (P.norm < 0 || P.norm > 3) return SD_ERR_ARG;
  P.newton_max = (opts && opts->newton_iters > 0) ? opts->newton_iters : 12;
  P.land_mask = opts ? opts->land_mask : nullptr;
  return SD_OK;
}

// words of a request's landing mask for pupil grids up to max_n
inline int mask_words(int max_n) { return (int)(((long long)max_n * max_n + 31) / 32); }

}  // namespace sd

extern "C" {

sd_status sd_dp_psf_trace(const sd_lens* const* lenses, int n_lenses,
                          const sd_dp_sensor* sensor, const sd_psf_request* req,
                          int n_req, const sd_trace_opts* opts, void* out,
                          int64_t* stats, void* stream) {
  SD_API_RANGE("sd_dp_psf_trace");
  using namespace sd;
  if (!opts || !out || (n_req > 0 && !req) || n_req < 0) return SD_ERR_ARG;
  if (n_req == 0) return SD_OK;
  TraceParams P;
  std::memset(&P, 0, sizeof P);
  sd_status st = fill_params(P, lenses, n_lenses, sensor, opts);
  if (st != SD_OK) return st;
  if (opts->mode != SD_BIN_HARD && opts->mode != SD_BIN_BILINEAR) return SD_ERR_ARG;
  if (opts->out_dtype < SD_F32 || opts->out_dtype > SD_F16) return SD_ERR_ARG;
  int max_ks = opts->max_ks;
  int max_n = opts->max_n_grid > 0 ? opts->max_n_grid : 512;
  if (max_ks < 1 || !(max_ks & 1)) return SD_ERR_ARG;
  if (max_ks > 127 || max_n > 2048 || max_n < 2) return SD_ERR_UNSUPPORTED;
  P.req = req;
  P.n_req = n_req;
  P.max_n = max_n;
  P.max_ks = max_ks;
  P.out = out;
  P.stats = reinterpret_cast<long long*>(stats);
  P.mask_words = mask_words(max_n);
  size_t smem = trace_smem_bytes(max_n, max_ks);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int threads = 256;
#define SD_LAUNCH(MODE, T)                                                          \
  do {                                                                              \
    auto kfn = trace_bin_kernel<MODE, T>;                                           \
    SD_CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)smem));                                   \
    kfn<<<n_req, threads, smem, s>>>(P);                                            \
  } while (0)
  if (opts->mode == SD_BIN_HARD) {
    if (opts->out_dtype == SD_F32) SD_LAUNCH(0, float);
    else if (opts->out_dtype == SD_BF16) SD_LAUNCH(0, __nv_bfloat16);
    else SD_LAUNCH(0, __half);
  } else {
    if (opts->out_dtype == SD_F32) SD_LAUNCH(1, float);
    else if (opts->out_dtype == SD_BF16) SD_LAUNCH(1, __nv_bfloat16);
    else SD_LAUNCH(1, __half);
  }
#undef SD_LAUNCH
  return launch_status();
}

sd_status sd_dp_psf_map(const sd_lens* lens, const sd_dp_sensor* sensor,
                        const float* depth_m, int H, int W, double lambda_nm,
                        int n_grid, int ks, const sd_trace_opts* opts, void* out,
                        int64_t* stats, void* stream) {
  SD_API_RANGE("sd_dp_psf_map");
  using namespace sd;
  if (!lens || !opts || !out || !depth_m || H < 0 || W < 0) return SD_ERR_ARG;
  if ((long long)H * W > 0x7fffffffLL) return SD_ERR_UNSUPPORTED;
  if (H == 0 || W == 0) return SD_OK;
  if (!(lambda_nm > 0) || n_grid < 2 || ks < 1 || !(ks & 1)) return SD_ERR_ARG;
  if (ks > 127 || n_grid > 2048) return SD_ERR_UNSUPPORTED;
  if (opts->mode != SD_BIN_HARD && opts->mode != SD_BIN_BILINEAR) return SD_ERR_ARG;
  if (opts->out_dtype < SD_F32 || opts->out_dtype > SD_F16) return SD_ERR_ARG;
  TraceParams P;
  std::memset(&P, 0, sizeof P);
  const sd_lens* ls[1] = {lens};
  sd_status st = fill_params(P, ls, 1, sensor, opts);
  if (st != SD_OK) return st;
  P.land_mask = nullptr;  // the map path writes no landing mask
  P.req = nullptr;
  P.n_req = H * W;
  P.map_depth = depth_m;
  P.map_H = H;
  P.map_W = W;
  P.map_lambda_nm = lambda_nm;
  P.map_n = n_grid;
  P.map_ks = ks;
  P.max_n = n_grid;
  P.max_ks = ks;
  P.out = out;
  P.stats = reinterpret_cast<long long*>(stats);
  size_t smem = trace_smem_bytes(n_grid, ks);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
#define SD_LAUNCH(MODE, T)                                                          \
  do {                                                                              \
    auto kfn = trace_bin_kernel<MODE, T>;                                           \
    SD_CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)smem));                                   \
    kfn<<<H * W, 256, smem, s>>>(P);                                                \
  } while (0)
  if (opts->mode == SD_BIN_HARD) {
    if (opts->out_dtype == SD_F32) SD_LAUNCH(0, float);
    else if (opts->out_dtype == SD_BF16) SD_LAUNCH(0, __nv_bfloat16);
    else SD_LAUNCH(0, __half);
  } else {
    if (opts->out_dtype == SD_F32) SD_LAUNCH(1, float);
    else if (opts->out_dtype == SD_BF16) SD_LAUNCH(1, __nv_bfloat16);
    else SD_LAUNCH(1, __half);
  }
#undef SD_LAUNCH
  return launch_status();
}

sd_status sd_dev_math_check(const float* a, const float* b, int n, float* quot,
                            float* root, void* stream) {
  using namespace sd;
  if (n < 0 || (n > 0 && (!a || !b || !quot || !root))) return SD_ERR_ARG;
  if (n == 0) return SD_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  math_check_kernel<<<(n + 255) / 256, 256, 0, s>>>(a, b, n, quot, root);
  return launch_status();
}

sd_status sd_dp_trace_hits(const sd_lens* lens, const sd_dp_sensor* sensor,
                           const sd_psf_request* req_host, const sd_trace_opts* opts,
                           float* rec, int max_rays, int32_t* n_rays, void* stream) {
  using namespace sd;
  if (!lens || !req_host || !rec || !n_rays || max_rays < 0) return SD_ERR_ARG;
  TraceParams P;
  std::memset(&P, 0, sizeof P);
  const sd_lens* ls[1] = {lens};
  sd_status st = fill_params(P, ls, 1, sensor, opts);
  if (st != SD_OK) return st;
  if (req_host->n_grid < 2 || req_host->n_grid > 2048) return SD_ERR_ARG;
  if (req_host->ks < 1 || !(req_host->ks & 1)) return SD_ERR_ARG;
  P.max_n = req_host->n_grid;
  P.max_ks = req_host->ks;
  P.rec = rec;
  P.max_rays = max_rays;
  P.n_rays = n_rays;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  sd_psf_request q = *req_host;
  q.lens = 0;  // the request is passed by value
  size_t smem = table_bytes(P.max_n);
  SD_CUDA_TRY(cudaFuncSetAttribute(trace_hits_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  trace_hits_kernel<<<1, 256, smem, s>>>(P, q);
  return launch_status();
}

}  // extern "C"

namespace sd {

// ---------------------------------------------------------------------------
// Adjoint trace (reverse mode by hand), bilinear splat, frozen decisions.
//
// Per ray the loss is  L = scale * sum_taps G[side][tap] w_tap(fx, fy)  with
// the bilinear weights of the landing point (Eq. 3 with unit energy split
// over the four nearest pixel centres) and scale = 1 (SD_NORM_NONE) or
// 1 / launched rays (SD_NORM_PER_RAY).  The ray is traced forward again
// (recompute instead of storing rays between passes), then swept backward:
// sensor propagation, and per surface Snell's law, the unit normal, the
// implicit-function derivative of the intersection (the Newton iteration is
// not unrolled: dt = -(grad Phi . dP) / (grad Phi . d) at convergence with
// Phi = z - sag(x^2 + y^2)), and the transfer by the thickness.  Ray
// generation is frozen; discrete decisions (reached, side, splat base pixel)
// are those of the forward pass.  Parameters per surface: curvature, conic,
// a4..a12, thickness after the surface (the last one is the sensor
// distance).
// ---------------------------------------------------------------------------
constexpr int NPAR_SURF = 8;

// Reverse sweep of one ray (V = float) or of two rays (V = float2, packed
// two-lane instructions; KS(s) yields the surface constants).  The forward
// pass kept only t at every surface
// and the hit point at the last one: going backwards, the incoming direction
// at a surface follows from its outgoing one by inverting Snell's law at the
// hit point (cos t_t = n . d_out, sin^2 t_i = sin^2 t_t / e^2, d_in =
// (d_out - g n) / e), and the previous hit point is P - t d_in (plus the
// thickness), so no per-surface state is stored.  `emit(s, v)` receives the
// 8 parameter adjoints of surface s (v[7] = thickness after it) and is
// called by every lane of the warp for s = n-1 .. 0.
template <class V, class KS, class Emit>
__device__ __forceinline__ void adjoint_ray(int n, const KS& ks_of, const AdjStateV<V>& sv,
                                            V dfx, V dfy, V dfz, V xb, V yb, Emit emit) {
  const V one = vb<V>(1.f), two = vb<V>(2.f), m2 = vb<V>(-2.f), mone = vb<V>(-1.f);
  V Px = sv.px, Py = sv.py, Pz = sv.pz;  // hit point at surface s
  V ox = dfx, oy = dfy, oz = dfz;        // direction leaving surface s
  // sensor: x_s = X + tau dx, tau = -Z / dz with Z the last hit moved to
  // sensor-local z
  const V Z = vadd(Pz, ks_of(n - 1).negt);
  const V tau = div_nr(vneg(Z), dfz);
  const V taub = vfma(yb, dfy, vmul(xb, dfx));
  V Pbx = xb, Pby = yb, Pbz = div_nr(vneg(taub), dfz);
  V dbx = vmul(xb, tau), dby = vmul(yb, tau), dbz = div_nr(vmul(taub, Z), vmul(dfz, dfz));
  V tcarry = vneg(Pbz);  // adjoint of the thickness after surface s
  for (int s = n - 1; s >= 0; --s) {
    const SurfK<V>& S = ks_of(s);
    const V t = sv.t[s];
    V v[NPAR_SURF];
#pragma unroll
    for (int j = 0; j < NPAR_SURF; ++j) v[j] = vb<V>(0.f);
    v[7] = tcarry;
    V ix = ox, iy = oy, iz = oz;  // direction arriving at the surface
    V ibx, iby, ibz;              // adjoint of the incoming direction
    V gx = vb<V>(0.f), gy = vb<V>(0.f), gz = one;  // grad Phi at the hit
    const V u = vfma(Py, Py, vmul(Px, Px));
    if (S.kind & K_REFRACT) {
      const V q = sqrt_nr(vfma(S.nkc2, u, one));
      const V iq = div_nr(one, q), iq3 = vmul(vmul(iq, iq), iq);
      // S1 = dsag/du = c / (2q) + sum_j (j+2) a_j u^(j+1)
      V up = one, S1 = vmul(S.halfc, iq), dS1 = vmul(S.qkc3, iq3);
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        dS1 = vfma(S.dda[j], up, dS1);  // (j+2)(j+1) a_j u^j
        up = vmul(up, u);
        S1 = vfma(S.da[j], up, S1);     // (j+2) a_j u^(j+1)
      }
      gx = vmul(vmul(m2, Px), S1);
      gy = vmul(vmul(m2, Py), S1);
      const V imn = rsqrt_refined(vfma(gy, gy, vfma(gx, gx, one)));
      const V nx = vmul(gx, imn), ny = vmul(gy, imn), nz = imn;
      // Snell: dout = e din + g n, g = (1 - e^2) / (ct + e cosi)
      const V ct = vfma(nz, oz, vfma(ny, oy, vmul(nx, ox)));
      const V cosi = sqrt_nr(vfma(vfma(ct, ct, mone), S.ie2, one));
      const V D = vfma(S.e, cosi, ct);
      const V g = div_nr(S.om, D), ng = vneg(g);
      ix = vmul(vfma(ng, nx, ox), S.ie);
      iy = vmul(vfma(ng, ny, oy), S.ie);
      iz = vmul(vfma(ng, nz, oz), S.ie);
      ibx = vmul(S.e, dbx);
      iby = vmul(S.e, dby);
      ibz = vmul(S.e, dbz);
      const V gb = vfma(dbz, nz, vfma(dby, ny, vmul(dbx, nx)));
      V nbx = vmul(g, dbx), nby = vmul(g, dby), nbz = vmul(g, dbz);
      const V Db = div_nr(vmul(gb, ng), D);
      const V k2b = div_nr(Db, vmul(two, ct));
      const V cosib = vfma(vmul(vmul(two, S.e2), k2b), cosi, vmul(Db, S.e));
      nbx = vfma(cosib, ix, nbx);
      nby = vfma(cosib, iy, nby);
      nbz = vfma(cosib, iz, nbz);
      ibx = vfma(cosib, nx, ibx);
      iby = vfma(cosib, ny, iby);
      ibz = vfma(cosib, nz, ibz);
      // n = m / |m|,  m = (-2 Px S1, -2 Py S1, 1)
      const V nnd = vneg(vfma(nz, nbz, vfma(ny, nby, vmul(nx, nbx))));
      const V mbx = vmul(vfma(nx, nnd, nbx), imn), mby = vmul(vfma(ny, nnd, nby), imn);
      const V S1b = vmul(m2, vfma(Py, mby, vmul(Px, mbx)));
      const V m2S1 = vmul(m2, S1);
      Pbx = vfma(m2S1, mbx, Pbx);
      Pby = vfma(m2S1, mby, Pby);
      const V ub = vmul(S1b, dS1);
      Pbx = vfma(vmul(two, Px), ub, Pbx);
      Pby = vfma(vmul(two, Py), ub, Pby);
      v[0] = vfma(S1b, vmul(vb<V>(0.5f), vfma(vmul(S.kc2, u), iq3, iq)), v[0]);
      v[1] = vfma(S1b, vmul(vmul(S.qc3, u), iq3), v[1]);
      up = u;
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        v[2 + j] = vfma(vmul(S1b, vb<V>((float)(j + 2))), up, v[2 + j]);  // u^(j+1)
        up = vmul(up, u);
      }
    } else {
      ibx = dbx;
      iby = dby;
      ibz = dbz;
    }
    // hit P = o + t din
    V obx = Pbx, oby = Pby, obz = Pbz;
    ibx = vfma(t, Pbx, ibx);
    iby = vfma(t, Pby, iby);
    ibz = vfma(t, Pbz, ibz);
    const V tb = vfma(Pbz, iz, vfma(Pby, iy, vmul(Pbx, ix)));
    // implicit intersection Phi(o + t din; theta) = 0
    const V lam = div_nr(vneg(tb), vfma(gz, iz, vfma(gy, iy, vmul(gx, ix))));
    obx = vfma(lam, gx, obx);
    oby = vfma(lam, gy, oby);
    obz = vfma(lam, gz, obz);
    const V lt = vmul(lam, t);
    ibx = vfma(lt, gx, ibx);
    iby = vfma(lt, gy, iby);
    ibz = vfma(lt, gz, ibz);
    if (S.kind & K_REFRACT) {
      const V q = sqrt_nr(vfma(S.nkc2, u, one));
      const V Sc = div_nr(vmul(S.c, u), vadd(one, q));  // conic part of the sag
      const V nli = vneg(div_nr(vmul(vb<V>(0.5f), lam), q));  // -lam / (2q)
      // Phi = z - sag:  dPhi/dc = -(u + (1+k) Sc^2) / (2q), dPhi/dk = -c Sc^2 / (2q),
      // dPhi/da_j = -u^(j+2)
      const V Sc2 = vmul(Sc, Sc);
      v[0] = vfma(nli, vfma(S.kk, Sc2, u), v[0]);
      v[1] = vfma(nli, vmul(S.c, Sc2), v[1]);
      const V nlam = vneg(lam);
      V up = vmul(u, u);
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        v[2 + j] = vfma(nlam, up, v[2 + j]);
        up = vmul(up, u);
      }
    }
    emit(s, v);
    // transfer: o_s = (P_{s-1}.x, P_{s-1}.y, P_{s-1}.z - T_{s-1})
    if (s > 0) {
      Pbx = obx;
      Pby = oby;
      Pbz = obz;
      tcarry = vneg(obz);
      dbx = ibx;
      dby = iby;
      dbz = ibz;
      const V nt = vneg(t);
      Px = vfma(nt, ix, Px);
      Py = vfma(nt, iy, Py);
      Pz = vsub(vfma(nt, iz, Pz), ks_of(s - 1).negt);
      ox = ix;
      oy = iy;
      oz = iz;
    }
  }
}

// Sum over the 32 lanes of a warp of 8 values per lane, as a reduce-scatter:
// on return, lane l holds the warp total of value (l >> 2) & 7 when
// (l & 3) == 0 (each exchange halves the values a lane carries).
__device__ __forceinline__ float warp_sum8(const float (&v)[NPAR_SURF], int lane) {
  float a[4], b[2], c;
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float send = h16 ? v[i] : v[i + 4];
    float keep = h16 ? v[i + 4] : v[i];
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  // a[i] holds value i + 4 * h16
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    float send = h8 ? a[i] : a[i + 2];
    float keep = h8 ? a[i + 2] : a[i];
    b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  // b[i] holds value i + 2 * h8 + 4 * h16
  {
    float send = h4 ? b[0] : b[1];
    float keep = h4 ? b[1] : b[0];
    c = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  // c holds value h4 + 2 * h8 + 4 * h16, summed over the lanes that differ
  // only in bits 2..4; finish over bits 0..1
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

// One block per request; per-request gradient partials greq[r][32*8].  The
// warps of a block run their rays' reverse sweeps in lockstep; after each
// surface the warp's 8 parameter adjoints are summed across its lanes
// (reduce-scatter) and added by one lane per parameter to the warp's row of
// a shared accumulator; the rows are added in warp order at the end (fixed
// order: deterministic).
// Three blocks per SM (80 registers, a few spilled): more warps to hide the
// sweep's dependent chains and the ray rounds' block barriers than two.
template <int NT>
__global__ void __launch_bounds__(NT, 3) trace_adj_kernel(TraceParams P, const float* __restrict__ G,
                                                       float* __restrict__ greq,
                                                       long long* __restrict__ swept) {
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ReqCtx ctx;
  __shared__ float s_acc[NW][SD_MAX_SURFACES][NPAR_SURF];
  __shared__ int s_swept[2];  // rays with a contribution, ray slots that ran the sweep
  __shared__ SurfK<float2> s_surf[SD_MAX_SURFACES];
  int* prefix = reinterpret_cast<int*>(smem);
  int* lo = prefix + (P.max_n + 1);
  float* Gs = reinterpret_cast<float*>(smem + table_bytes(P.max_n));
  const int r = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const sd_psf_request q = request_of(P, r);
  for (int i = threadIdx.x; i < NW * SD_MAX_SURFACES * NPAR_SURF; i += NT)
    (&s_acc[0][0][0])[i] = 0.f;
  if (threadIdx.x < 2) s_swept[threadIdx.x] = 0;
  setup_request(P, q, ctx, prefix, lo);
  const int ks = ctx.ks, ks2 = ks * ks, pp = (ks - 1) >> 1;
  bool nz = false;
  for (int i = threadIdx.x; i < 2 * ks2; i += NT) {
    const float g = G[q.out_offset + i];
    Gs[i] = g;
    nz = nz || g != 0.f;
  }
  // a request whose gradient patch is zero has an exactly zero parameter
  // gradient (every ray's splat gradient vanishes): no ray is traced again
  if (!__syncthreads_or(nz)) {
    for (int i = threadIdx.x; i < SD_MAX_SURFACES * NPAR_SURF; i += NT)
      greq[(size_t)r * SD_MAX_SURFACES * NPAR_SURF + i] = 0.f;
    if (swept && threadIdx.x < 2) swept[2 * (size_t)r + threadIdx.x] = 0;
    return;
  }
  const SensorF S = P.sen;
  const int total = ctx.N ? ctx.total : 0;
  const float scale = (P.norm == SD_NORM_PER_RAY) ? (total > 0 ? 1.f / (float)total : 0.f) : 1.f;
  const int n = ctx.N ? c_lens[ctx.slot].n : 0;
  for (int sf = threadIdx.x; sf < n; sf += NT)
    s_surf[sf] = pair_consts(surf_consts(c_lens[ctx.slot].s[sf], ctx.eta[sf], ctx.omeg2[sf]));
  __syncthreads();
  auto ks_of = [&](int sf) -> const SurfK<float2>& { return s_surf[sf]; };
  AdjStateV<float2> sv;
  int row0 = 0, row1 = 0;
  // A thread takes two rays a round (k and k + NT of the round's rays) and
  // traces and sweeps them as a packed pair.  With a landing mask the rays
  // whose bit is set are taken in ray order from a ring queue that warp 0
  // refills 32 mask words at a time, 2 NT per round, so that every warp but
  // the request's last is full; without one, every ray (2 NT consecutive
  // rays per round).
  constexpr int QCAP = 2048;  // > 2 NT - 1 + 32 * 32: a refill never wraps onto live entries
  static_assert(QCAP > 2 * NT - 1 + 32 * 32, "ray queue too small");
  __shared__ int s_q[QCAP];
  __shared__ int s_head, s_qn, s_wpos;
  const unsigned* mw = P.land_mask ? P.land_mask + (size_t)r * P.mask_words : nullptr;
  const int nwords = (total + 31) >> 5;
  if (threadIdx.x == 0) s_head = s_qn = s_wpos = 0;
  int take = 0;  // rays handed out in the previous round
  for (int base = 0;; base += 2 * NT) {
    int k0, k1;
    if (mw) {
      __syncthreads();  // every thread has its previous ray
      if (warp == 0) {
        int head = (s_head + take) & (QCAP - 1), qn = s_qn - take, wpos = s_wpos;
        while (qn < 2 * NT && wpos < nwords) {
          const int wi = wpos + lane;
          unsigned m = wi < nwords && SD_CHECK(wi, P.mask_words) ? mw[wi] : 0u;
          const int c = __popc(m);
          int pre = c;  // inclusive prefix of the counts over the lanes
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += t;
          }
          const int all = __shfl_sync(0xffffffffu, pre, 31);
          int pos = head + qn + pre - c;
          while (m) {
            s_q[pos & (QCAP - 1)] = (wi << 5) + __ffs(m) - 1;
            m &= m - 1;
            ++pos;
          }
          qn += all;
          wpos += 32;
        }
        if (lane == 0) {
          s_head = head;
          s_qn = qn;
          s_wpos = wpos;
        }
      }
      __syncthreads();
      const int qn = s_qn;
      if (qn == 0) break;
      take = min(qn, 2 * NT);
      const int t0 = threadIdx.x, t1 = threadIdx.x + NT;
      k0 = t0 < take ? s_q[(s_head + t0) & (QCAP - 1)] : total;
      k1 = t1 < take ? s_q[(s_head + t1) & (QCAP - 1)] : total;
    } else {
      if (base >= total) break;
      k0 = base + threadIdx.x;
      k1 = k0 + NT;
    }
    float2 x = make_float2(0.f, 0.f), y = x, z = x, dx = x, dy = x,
           dz = make_float2(1.f, 1.f);
    int2 st = make_int2(k0 < total ? (int)ST_OK : (int)ST_NONE,
                        k1 < total ? (int)ST_OK : (int)ST_NONE);
    if (k0 < total) {
      row0 = advance_row(prefix, k0, row0);
      make_ray_row(ctx, prefix, lo, k0, row0, x.x, y.x, z.x, dx.x, dy.x, dz.x);
    }
    if (k1 < total) {
      row1 = advance_row(prefix, k1, row1);
      make_ray_row(ctx, prefix, lo, k1, row1, x.y, y.y, z.y, dx.y, dy.y, dz.y);
    }
    if (k0 < total)
      st = trace_ray_v<true, float2>(n, ks_of, P.newton_max, st, x, y, z, dx, dy, dz, &sv);
    // the splat gradient of one ray (the forward's decisions)
    auto splat = [&](int stv, float xv, float yv, float dxv, float dzv, float& gfx, float& gfy) {
      gfx = gfy = 0.f;
      if (stv != ST_OK) return false;
      float fx = (xv - ctx.xc) * S.inv_ps + (float)pp;
      float fy = (yv - ctx.yc) * S.inv_ps + (float)pp;
      float af = floorf(fx + 0.5f), bf = floorf(fy + 0.5f);
      int side = dp_side(S, (fx - af) * S.ps, (fy - bf) * S.ps, tan_theta(dxv, dzv));
      if (side == 2) return false;
      float a0f = floorf(fx), b0f = floorf(fy);
      float wx = fx - a0f, wy = fy - b0f;
      int a0 = (int)a0f, b0 = (int)b0f;
      const float* Gp = Gs + side * ks2;
#pragma unroll
      for (int jy = 0; jy < 2; ++jy)
#pragma unroll
        for (int jx = 0; jx < 2; ++jx) {
          int aa = a0 + jx, bb = b0 + jy;
          if (aa < 0 || aa >= ks || bb < 0 || bb >= ks) continue;
          float gv = Gp[bb * ks + aa];
          gfx += gv * (jx ? 1.f : -1.f) * (jy ? wy : 1.f - wy);
          gfy += gv * (jy ? 1.f : -1.f) * (jx ? wx : 1.f - wx);
        }
      return gfx != 0.f || gfy != 0.f;
    };
    float gfx0, gfy0, gfx1, gfy1;
    const bool need0 = splat(st.x, x.x, y.x, dx.x, dz.x, gfx0, gfy0);
    const bool need1 = splat(st.y, x.y, y.y, dx.y, dz.y, gfx1, gfy1);
    // the whole warp sweeps when any ray of it needs it; the other rays
    // contribute exact zeros (their values are selected away, never added)
    const unsigned nm0 = __ballot_sync(0xffffffffu, need0);
    const unsigned nm1 = __ballot_sync(0xffffffffu, need1);
    if (!(nm0 | nm1)) continue;
    if (lane == 0) {
      atomicAdd(&s_swept[0], __popc(nm0) + __popc(nm1));
      atomicAdd(&s_swept[1], 64);
    }
    if (!(need0 && need1)) {
      // a harmless state for the rays without a contribution
      const float2 zero = make_float2(0.f, 0.f);
      const M2 keep{need0, need1};
      sv.px = sel(keep, sv.px, zero);
      sv.py = sel(keep, sv.py, zero);
      sv.pz = sel(keep, sv.pz, zero);
      for (int s2 = 0; s2 < n; ++s2) sv.t[s2] = sel(keep, sv.t[s2], zero);
      dx = sel(keep, dx, zero);
      dy = sel(keep, dy, zero);
      dz = sel(keep, dz, make_float2(1.f, 1.f));
    }
    const float gs = scale * S.inv_ps;
    adjoint_ray<float2>(n, ks_of, sv, dx, dy, dz, make_float2(gs * gfx0, gs * gfx1),
                        make_float2(gs * gfy0, gs * gfy1), [&](int s2, float2 (&v)[NPAR_SURF]) {
                          // the pair's two rays added first (ray k, then k + NT)
                          float w[NPAR_SURF];
#pragma unroll
                          for (int j2 = 0; j2 < NPAR_SURF; ++j2)
                            w[j2] = (need0 ? v[j2].x : 0.f) + (need1 ? v[j2].y : 0.f);
                          const float tot = warp_sum8(w, lane);
                          if ((lane & 3) == 0) s_acc[warp][s2][(lane >> 2) & 7] += tot;
                        });
  }
  __syncthreads();
  // per-request partials: warps added in order
  for (int i = threadIdx.x; i < SD_MAX_SURFACES * NPAR_SURF; i += NT) {
    const int s2 = i / NPAR_SURF, j2 = i - s2 * NPAR_SURF;
    float a = 0.f;
    if (s2 < n)
      for (int w = 0; w < NW; ++w) a += s_acc[w][s2][j2];
    greq[(size_t)r * SD_MAX_SURFACES * NPAR_SURF + i] = a;
  }
  if (swept && threadIdx.x < 2) swept[2 * (size_t)r + threadIdx.x] = s_swept[threadIdx.x];
}

// Sums the per-request partials of each lens: four contiguous request
// ranges per parameter, added in range order (deterministic).
__global__ void __launch_bounds__(1024) grad_lens_reduce(const float* __restrict__ greq,
                                                         const sd_psf_request* req, int n_req,
                                                         int n_lenses, float* __restrict__ glens) {
  constexpr int NP = SD_MAX_SURFACES * NPAR_SURF;  // 256
  __shared__ float part[4][NP];
  const int li = blockIdx.x, pidx = threadIdx.x % NP, ch = threadIdx.x / NP;
  const int r0 = (int)((long long)n_req * ch / 4), r1 = (int)((long long)n_req * (ch + 1) / 4);
  float a = 0.f;
#pragma unroll 8
  for (int r = r0; r < r1; ++r)
    if (__ldg(&req[r].lens) == li) a += __ldg(&greq[(size_t)r * NP + pidx]);
  part[ch][pidx] = a;
  __syncthreads();
  if (ch == 0)
    glens[(size_t)li * NP + pidx] = ((part[0][pidx] + part[1][pidx]) + part[2][pidx]) + part[3][pidx];
}

}  // namespace sd

extern "C" sd_status sd_dp_psf_trace_mask_bytes(int n_req, int max_n_grid, size_t* bytes) {
  if (!bytes || n_req < 0 || max_n_grid < 0 || max_n_grid > 2048) return SD_ERR_ARG;
  const int max_n = max_n_grid > 0 ? max_n_grid : 512;
  *bytes = (size_t)n_req * sd::mask_words(max_n) * 4;
  return SD_OK;
}

extern "C" sd_status sd_dp_psf_trace_backward(const sd_lens* const* lenses, int n_lenses,
                                              const sd_dp_sensor* sensor,
                                              const sd_psf_request* req, int n_req,
                                              const sd_trace_opts* opts, const float* grad_out,
                                              float* grad_req, float* grad_lens,
                                              int64_t* swept, void* stream) {
  SD_API_RANGE("sd_dp_psf_trace_backward");
  using namespace sd;
  if (!opts || !grad_out || !grad_req || n_req < 0 || (n_req > 0 && !req)) return SD_ERR_ARG;
  TraceParams P;
  std::memset(&P, 0, sizeof P);
  sd_status st = fill_params(P, lenses, n_lenses, sensor, opts);
  if (st != SD_OK) return st;
  if (opts->mode != SD_BIN_BILINEAR) return SD_ERR_UNSUPPORTED;
  if (opts->norm != SD_NORM_NONE && opts->norm != SD_NORM_PER_RAY) return SD_ERR_UNSUPPORTED;
  if (opts->out_dtype != SD_F32) return SD_ERR_UNSUPPORTED;
  int max_ks = opts->max_ks;
  int max_n = opts->max_n_grid > 0 ? opts->max_n_grid : 512;
  if (max_ks < 1 || !(max_ks & 1)) return SD_ERR_ARG;
  if (max_ks > 127 || max_n > 2048 || max_n < 2) return SD_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (n_req == 0) {
    if (grad_lens)
      SD_CUDA_TRY(cudaMemsetAsync(grad_lens, 0,
                                  (size_t)n_lenses * SD_MAX_SURFACES * NPAR_SURF * 4, s));
    return SD_OK;
  }
  P.req = req;
  P.n_req = n_req;
  P.max_n = max_n;
  P.max_ks = max_ks;
  P.mask_words = mask_words(max_n);
  size_t smem = table_bytes(max_n) + (size_t)2 * max_ks * max_ks * 4;
  // Surface count read at run time; the forward keeps one t per surface (a
  // local array) and the reverse sweep rebuilds the rest.  Variants with the
  // count fixed at compile time and the whole per-surface state in registers
  // needed 130-190 registers per thread and measured slower.
  constexpr int NT = 256;
  void (*k)(TraceParams, const float*, float*, long long*) = trace_adj_kernel<NT>;
  SD_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k<<<n_req, NT, smem, s>>>(P, grad_out, grad_req, reinterpret_cast<long long*>(swept));
  st = launch_status();
  if (st != SD_OK) return st;
  if (grad_lens) {
    grad_lens_reduce<<<n_lenses, 1024, 0, s>>>(grad_req, req, n_req, n_lenses, grad_lens);
    st = launch_status();
  }
  return st;
}

namespace sd {

// ---------------------------------------------------------------------------
// Batched trace of uneven requests in one persistent launch.
//
// prep_kernel (one block per request): FP64 set-up of the request (the same
//   prologue as the per-request kernel), its in-pupil ray count, and its
//   split into work items of whole pupil rows (about rays_per_chunk rays);
//   zeroes the request's count patch, statistics and completion counter.
// item_scan_kernel: exclusive prefix of the item counts (item -> request).
// batched_trace_kernel: a fixed grid of blocks; block b processes the
//   contiguous item range [b M / G, (b+1) M / G).  While consecutive items
//   belong to one request the block accumulates them in its shared patch; on
//   a change of request (and at the end) it adds the patch to the request's
//   u32 counts with integer atomics (order-independent: deterministic),
//   then counts its items on the request's completion counter.  The block
//   that completes a request normalises and stores it (no waiting on other
//   blocks).  Hard binning only.
// ---------------------------------------------------------------------------
struct BatchCtx {
  ReqCtx c;
  int n_items, rows_per_item;
  long long off;
};

struct BatchWs {
  BatchCtx* ctx;       // [n_req]
  int* item_start;     // [n_req + 1]
  unsigned* done;      // [n_req]
  unsigned* counts;    // [total elements], u32
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__host__ __device__ inline BatchWs batch_ws(void* base, int n_req) {
  BatchWs w;
  char* p = reinterpret_cast<char*>(base);
  w.ctx = reinterpret_cast<BatchCtx*>(p);
  p += align256(sizeof(BatchCtx) * (size_t)n_req);
  w.item_start = reinterpret_cast<int*>(p);
  p += align256(sizeof(int) * ((size_t)n_req + 1));
  w.done = reinterpret_cast<unsigned*>(p);
  p += align256(sizeof(unsigned) * (size_t)n_req);
  w.counts = reinterpret_cast<unsigned*>(p);
  return w;
}

__host__ __device__ inline size_t batch_ws_bytes(int n_req, long long total_elems) {
  return align256(sizeof(BatchCtx) * (size_t)n_req) + align256(sizeof(int) * ((size_t)n_req + 1)) +
         align256(sizeof(unsigned) * (size_t)n_req) + sizeof(unsigned) * (size_t)total_elems;
}

__global__ void __launch_bounds__(128) prep_kernel(TraceParams P, BatchWs W, int rays_per_item,
                                                   long long total_elems) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ReqCtx ctx;
  int* prefix = reinterpret_cast<int*>(smem);
  int* lo = prefix + (P.max_n + 1);
  const int r = blockIdx.x;
  const sd_psf_request q = request_of(P, r);
  setup_request(P, q, ctx, prefix, lo);
  const int ks2 = ctx.ks * ctx.ks;
  const bool fits = ctx.N && q.out_offset >= 0 && q.out_offset + 2LL * ks2 <= total_elems;
  if (threadIdx.x == 0) {
    BatchCtx b;
    b.c = ctx;
    if (!fits) b.c.N = 0;
    b.rows_per_item = max(1, rays_per_item / max(1, ctx.N));
    b.n_items = fits ? (ctx.N + b.rows_per_item - 1) / b.rows_per_item : 0;
    b.off = q.out_offset;
    W.ctx[r] = b;
    W.item_start[r] = b.n_items;  // counts; scanned by item_scan_kernel
    W.done[r] = 0u;
  }
  if (fits)
    for (int i = threadIdx.x; i < 2 * ks2; i += blockDim.x) W.counts[q.out_offset + i] = 0u;
  // the items OR their rays' landing bits into the request's mask words
  if (fits && P.land_mask)
    for (int i = threadIdx.x; i < (ctx.total + 31) >> 5; i += blockDim.x)
      if (SD_CHECK(i, P.mask_words)) P.land_mask[(size_t)r * P.mask_words + i] = 0u;
  if (P.stats && threadIdx.x < SD_N_STATS)
    P.stats[(long long)r * SD_N_STATS + threadIdx.x] =
        threadIdx.x == SD_STAT_LAUNCHED && fits ? (long long)ctx.total : 0;
}

__global__ void __launch_bounds__(1024) item_scan_kernel(int* item_start, int n_req) {
  // single block exclusive scan, in place, item_start[n_req] = total
  __shared__ int s_carry, s_w[32];
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < n_req; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < n_req ? item_start[i] : 0;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int w = s_w[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += t;
      }
      s_w[lane] = w;
    }
    __syncthreads();
    int incl = x + (warp ? s_w[warp - 1] : 0) + s_carry;
    if (i < n_req) item_start[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) item_start[n_req] = s_carry;
}

// Adds the block's patch of request r to its counts; the block that
// completes the request's items normalises and stores it.
template <class OutT>
__device__ void batch_flush(const TraceParams& P, const BatchWs& W, int r, int items_here,
                            unsigned* patch, unsigned* s_stats, int* s_last, float* s_red) {
  const BatchCtx& B = W.ctx[r];
  const int ks = B.c.ks, ks2 = ks * ks;
  unsigned* cnt = W.counts + B.off;
  for (int i = threadIdx.x; i < 2 * ks2; i += blockDim.x) {
    unsigned v = patch[i];
    if (v) atomicAdd(&cnt[i], v);
    patch[i] = 0u;
  }
  if (P.stats && threadIdx.x < SD_N_STATS && threadIdx.x != SD_STAT_LAUNCHED) {
    unsigned v = s_stats[threadIdx.x];
    if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&P.stats[(long long)r * SD_N_STATS +
                                                                     threadIdx.x]),
                     (unsigned long long)v);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x < SD_N_STATS) s_stats[threadIdx.x] = 0u;
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(&W.done[r], (unsigned)items_here);
    *s_last = (prev + (unsigned)items_here == (unsigned)B.n_items);
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  // normalise (same arithmetic as the per-request kernel) and store
  float sl = 0.f, sr = 0.f;
  for (int i = threadIdx.x; i < ks2; i += blockDim.x) {
    sl += (float)__ldcg(&cnt[i]);
    sr += (float)__ldcg(&cnt[ks2 + i]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sl += __shfl_xor_sync(0xffffffffu, sl, o);
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s_red[warp] = sl;
    s_red[32 + warp] = sr;
  }
  __syncthreads();
  float SL = 0.f, SR = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    SL += s_red[w];
    SR += s_red[32 + w];
  }
  float scl = 1.f, scr = 1.f;
  if (P.norm == SD_NORM_JOINT) {
    float s = SL + SR;
    scl = scr = s > 0.f ? 1.f / s : 0.f;
  } else if (P.norm == SD_NORM_SEPARATE) {
    scl = SL > 0.f ? 1.f / SL : 0.f;
    scr = SR > 0.f ? 1.f / SR : 0.f;
  } else if (P.norm == SD_NORM_PER_RAY) {
    scl = scr = B.c.total > 0 ? 1.f / (float)B.c.total : 0.f;
  }
  for (int i = threadIdx.x; i < 2 * ks2; i += blockDim.x)
    store_out<OutT>(P.out, B.off + i, (float)__ldcg(&cnt[i]) * (i < ks2 ? scl : scr));
  __syncthreads();
}

template <class OutT>
__global__ void __launch_bounds__(1024) batched_trace_kernel(TraceParams P, BatchWs W, int n_req) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ReqCtx ctx;
  __shared__ unsigned s_stats[SD_N_STATS];
  __shared__ float s_red[64];
  __shared__ int s_last, s_rows, s_off;
  __shared__ SurfK<float2> s_surf[SD_MAX_SURFACES];
  int* prefix = reinterpret_cast<int*>(smem);
  int* lo = prefix + (P.max_n + 1);
  unsigned* patch = reinterpret_cast<unsigned*>(smem + table_bytes(P.max_n));
  auto ks_of = [&](int sf) -> const SurfK<float2>& { return s_surf[sf]; };
  const int M = W.item_start[n_req];
  const int G = gridDim.x, b = blockIdx.x;
  const int i0 = (int)((long long)M * b / G), i1 = (int)((long long)M * (b + 1) / G);
  for (int i = threadIdx.x; i < 2 * P.max_ks * P.max_ks; i += blockDim.x) patch[i] = 0u;
  if (threadIdx.x < SD_N_STATS) s_stats[threadIdx.x] = 0u;
  const SensorF S = P.sen;
  const int lane = threadIdx.x & 31;
  int cur = -1, items_here = 0;
  for (int it = i0; it < i1; ++it) {
    // request of item it: last r with item_start[r] <= it
    int a = 0, e = n_req;
    while (e - a > 1) {
      int m = (a + e) >> 1;
      if (W.item_start[m] <= it) a = m; else e = m;
    }
    const int r = a;
    if (r != cur) {
      __syncthreads();
      if (cur >= 0) batch_flush<OutT>(P, W, cur, items_here, patch, s_stats, &s_last, s_red);
      if (threadIdx.x == 0) ctx = W.ctx[r].c;
      cur = r;
      items_here = 0;
      __syncthreads();
      // the request's surface constants as pairs (read after the next barrier)
      for (int sf = threadIdx.x; sf < c_lens[ctx.slot].n; sf += blockDim.x)
        s_surf[sf] = pair_consts(surf_consts(c_lens[ctx.slot].s[sf], ctx.eta[sf], ctx.omeg2[sf]));
    }
    ++items_here;
    // rows of this item and their in-pupil spans
    const int N = ctx.N, ks = ctx.ks, ks2 = ks * ks, pp = (ks - 1) >> 1;
    const int rpi = W.ctx[r].rows_per_item;
    const int row0 = (it - W.item_start[r]) * rpi, row1 = min(N, row0 + rpi);
    const int nrows = row1 - row0;
    for (int j = threadIdx.x; j < nrows; j += blockDim.x) {
      int c, l;
      row_span(N, row0 + j, &c, &l);
      prefix[j + 1] = c;
      lo[j] = l;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      int carry = 0;
      for (int base = 0; base < nrows; base += 32) {
        int j = base + lane;
        int v = j < nrows ? prefix[j + 1] : 0;
        for (int o = 1; o < 32; o <<= 1) {
          int t = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += t;
        }
        if (j < nrows) prefix[j + 1] = v + carry;
        carry += __shfl_sync(0xffffffffu, v, 31);
      }
      if (lane == 0) {
        prefix[0] = 0;
        s_rows = carry;
      }
    }
    if (threadIdx.x == 0) s_off = 0;
    __syncthreads();
    const int total = s_rows;
    if (P.land_mask) {
      // the request's rays before this item (its rows above row0): the
      // item's first ray index in the request's landing mask
      int c_above = 0;
      for (int j = threadIdx.x; j < row0; j += blockDim.x) {
        int c, l;
        row_span(N, j, &c, &l);
        c_above += c;
      }
      if (c_above) atomicAdd(&s_off, c_above);
      __syncthreads();
    }
    const int ray0 = s_off;
    unsigned c_reached = 0, c_vign = 0, c_other = 0, c_l = 0, c_r = 0, c_miss = 0, c_clip = 0;
    // bins ray k of the item (one of a set of blockDim.x consecutive rays,
    // every thread calls it for each set), as trace_bin_kernel does
    auto bin = [&](int k, int st, float x, float y, float dx, float dz) {
      int key = -1;
      bool land = false;
      if (k < total) {
        if (st == ST_OK) {
          ++c_reached;
          float fx = (x - ctx.xc) * S.inv_ps + (float)pp;
          float fy = (y - ctx.yc) * S.inv_ps + (float)pp;
          float af = floorf(fx + 0.5f), bf = floorf(fy + 0.5f);
          int side = dp_side(S, (fx - af) * S.ps, (fy - bf) * S.ps, tan_theta(dx, dz));
          bool inpatch = af >= 0.f && af < (float)ks && bf >= 0.f && bf < (float)ks;
          if (!inpatch) ++c_clip;
          else if (side == 2) ++c_miss;
          else if (side == 0) ++c_l;
          else ++c_r;
          if (inpatch && side < 2) key = side * ks2 + (int)bf * ks + (int)af;
          land = side != 2 && af >= -1.f && af <= (float)ks && bf >= -1.f && bf <= (float)ks;
        } else if (st == ST_CLIP) {
          ++c_vign;
        } else {
          ++c_other;
        }
      }
      if (P.land_mask) {
        // the warp's 32 rays start at request ray g0, which need not be a
        // word boundary: their bits go to words g0 / 32 and the next
        const unsigned bits = __ballot_sync(0xffffffffu, land);
        const int g0 = ray0 + k - lane, w0 = g0 >> 5, sh = g0 & 31;
        if (lane == 0 && bits) {
          unsigned* mr = P.land_mask + (size_t)r * P.mask_words;
          if (SD_CHECK(w0, P.mask_words)) atomicOr(mr + w0, bits << sh);
          const unsigned hi = sh ? bits >> (32 - sh) : 0u;
          if (hi && SD_CHECK(w0 + 1, P.mask_words)) atomicOr(mr + w0 + 1, hi);
        }
      }
      unsigned m = __match_any_sync(0xffffffffu, key);
      if (key >= 0 && lane == __ffs(m) - 1) atomicAdd(&patch[key], (unsigned)__popc(m));
    };
    // rays k and k + blockDim.x of the item (k grows within the item: each
    // advances its own row) traced together as a packed pair
    const int NT = blockDim.x;
    int rw0 = 0, rw1 = 0;
    const int nsurf = c_lens[ctx.slot].n;
    for (int base = 0; base < total; base += 2 * NT) {
      const int k0 = base + threadIdx.x, k1 = k0 + NT;
      float2 x = make_float2(0.f, 0.f), y = x, z = x, dx = x, dy = x,
             dz = make_float2(1.f, 1.f);
      int2 st = make_int2(k0 < total ? (int)ST_OK : (int)ST_NONE,
                          k1 < total ? (int)ST_OK : (int)ST_NONE);
      if (k0 < total) {
        rw0 = advance_row(prefix, k0, rw0);
        pupil_ray(ctx, lo[rw0] + (k0 - prefix[rw0]), row0 + rw0, x.x, y.x, z.x, dx.x, dy.x,
                  dz.x);
      }
      if (k1 < total) {
        rw1 = advance_row(prefix, k1, rw1);
        pupil_ray(ctx, lo[rw1] + (k1 - prefix[rw1]), row0 + rw1, x.y, y.y, z.y, dx.y, dy.y,
                  dz.y);
      }
      if (k0 < total)
        st = trace_ray_v<false, float2>(nsurf, ks_of, P.newton_max, st, x, y, z, dx, dy, dz,
                                        nullptr);
      bin(k0, st.x, x.x, y.x, dx.x, dz.x);
      bin(k1, st.y, x.y, y.y, dx.y, dz.y);
    }
    atomicAdd(&s_stats[SD_STAT_REACHED], c_reached);
    atomicAdd(&s_stats[SD_STAT_VIGNETTED], c_vign);
    atomicAdd(&s_stats[SD_STAT_OTHER], c_other);
    atomicAdd(&s_stats[SD_STAT_L], c_l);
    atomicAdd(&s_stats[SD_STAT_R], c_r);
    atomicAdd(&s_stats[SD_STAT_DP_MISSED], c_miss);
    atomicAdd(&s_stats[SD_STAT_CLIPPED], c_clip);
    __syncthreads();  // row tables are rewritten by the next item
  }
  __syncthreads();
  if (cur >= 0) batch_flush<OutT>(P, W, cur, items_here, patch, s_stats, &s_last, s_red);
}

size_t batched_smem_bytes(int max_n, int max_ks) {
  return table_bytes(max_n) + (size_t)2 * max_ks * max_ks * 4;
}

}  // namespace sd

extern "C" {

sd_status sd_dp_psf_trace_batched_workspace(int n_req, long long total_elems, size_t* bytes) {
  if (!bytes || n_req < 0 || total_elems < 0) return SD_ERR_ARG;
  *bytes = sd::batch_ws_bytes(n_req, total_elems);
  return SD_OK;
}

sd_status sd_dp_psf_trace_batched(const sd_lens* const* lenses, int n_lenses,
                                  const sd_dp_sensor* sensor, const sd_psf_request* req,
                                  int n_req, const sd_trace_opts* opts,
                                  const sd_batch_config* cfg, void* out, long long total_elems,
                                  int64_t* stats, void* workspace, size_t workspace_bytes,
                                  void* stream) {
  SD_API_RANGE("sd_dp_psf_trace_batched");
  using namespace sd;
  if (!opts || !out || n_req < 0 || (n_req > 0 && !req) || total_elems < 0) return SD_ERR_ARG;
  if (n_req == 0) return SD_OK;
  TraceParams P;
  std::memset(&P, 0, sizeof P);
  sd_status st = fill_params(P, lenses, n_lenses, sensor, opts);
  if (st != SD_OK) return st;
  if (opts->mode != SD_BIN_HARD) return SD_ERR_UNSUPPORTED;
  if (opts->out_dtype < SD_F32 || opts->out_dtype > SD_F16) return SD_ERR_ARG;
  int max_ks = opts->max_ks;
  int max_n = opts->max_n_grid > 0 ? opts->max_n_grid : 512;
  if (max_ks < 1 || !(max_ks & 1)) return SD_ERR_ARG;
  if (max_ks > 127 || max_n > 2048 || max_n < 2) return SD_ERR_UNSUPPORTED;
  if (!workspace || workspace_bytes < batch_ws_bytes(n_req, total_elems)) return SD_ERR_ARG;
  sd_batch_config c{};
  if (cfg) c = *cfg;
  if (c.threads == 0) c.threads = 512;
  if (c.rays_per_item == 0) c.rays_per_item = 16384;
  if (c.blocks_per_sm == 0) c.blocks_per_sm = 1;
  if (c.threads % 32 || c.threads < 64 || c.threads > 1024 || c.rays_per_item < 1 ||
      c.blocks_per_sm < 1 || c.blocks_per_sm > 8)
    return SD_ERR_ARG;
  P.req = req;
  P.n_req = n_req;
  P.max_n = max_n;
  P.max_ks = max_ks;
  P.mask_words = mask_words(max_n);
  P.out = out;
  P.stats = reinterpret_cast<long long*>(stats);
  BatchWs W = batch_ws(workspace, n_req);  // u32 counts at the requests' output offsets
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  size_t psmem = table_bytes(max_n);
  SD_CUDA_TRY(cudaFuncSetAttribute(prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)psmem));
  prep_kernel<<<n_req, 128, psmem, s>>>(P, W, c.rays_per_item, total_elems);
  if ((st = launch_status()) != SD_OK) return st;
  item_scan_kernel<<<1, 1024, 0, s>>>(W.item_start, n_req);
  if ((st = launch_status()) != SD_OK) return st;
  int dev = 0, n_sm = 0;
  SD_CUDA_TRY(cudaGetDevice(&dev));
  SD_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  size_t smem = batched_smem_bytes(max_n, max_ks);
  int grid = n_sm * c.blocks_per_sm;
#define SD_BLAUNCH(T)                                                                    \
  do {                                                                                   \
    auto kfn = batched_trace_kernel<T>;                                                  \
    SD_CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                     (int)smem));                                        \
    kfn<<<grid, c.threads, smem, s>>>(P, W, n_req);                                      \
  } while (0)
  if (opts->out_dtype == SD_F32) SD_BLAUNCH(float);
  else if (opts->out_dtype == SD_BF16) SD_BLAUNCH(__nv_bfloat16);
  else SD_BLAUNCH(__half);
#undef SD_BLAUNCH
  return launch_status();
}

}  // extern "C"

SD_CHECK_TU(lens_trace)
