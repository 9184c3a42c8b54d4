// FP64 CPU oracle of the Sdirt dual-pixel (DP) simulator hot path.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// cpu_baseline / reference legs of bench.py may load this library.  It shares
// no code, header, table or constant with the CUDA library: its C interface is
// declared only here and mirrored by the ctypes wrapper in oracle/__init__.py.
//
// Everything is plain, slow and written step by step in the order of the
// paper (He et al., "Simulating Dual-Pixel Images From Ray Tracing For Depth
// Estimation", ICCV 2025):
//   * lens model: Tables S1/S2 columns (radius, thickness, nd/Vd, diameter,
//     conic, a4..a12); even-asphere sag.
//   * Sec. 3.1: ray set A from object point p to n entrance-pupil samples,
//     sequential refraction by Snell's law, landing point O and direction D.
//   * Sec. 3.1 Eq. (1)/(2): left/right sub-pixel test inside/outside the
//     microlens; Eq. (S1) pixel constants are passed in by the caller.
//   * Sec. 3.1 Eq. (3): PSF_L/PSF_R = sum of unit ray energies.
//   * Sec. 3.2: sum normalisation of the DP PSFs.
//   * Supplement "Local DP PSF convolution": per-pixel rendering with the
//     pixel's own flipped PSF on a replicate-padded image.
// Readings of points the paper leaves open are stated where they are used.
//
// Precision: FP64 throughout, except the per-pixel bank selection of the
// renderer (nearest field height, depth bracket), an integer decision that is
// taken in FP32 exactly as the GPU kernel takes it.
// Gradients: the same templated trace is run with forward-mode dual numbers
// (exact derivatives of the branch the real parts select).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// --------------------------------------------------------------------------
// Scalars: double, or a dual number carrying up to ND partial derivatives.
// --------------------------------------------------------------------------
constexpr int ND = 24;

struct Dual {
  double v;
  double d[ND];
  Dual() : v(0) { std::memset(d, 0, sizeof d); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof d); }  // NOLINT
};
inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r(a.v + b.v);
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r(a.v - b.v);
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
inline Dual operator-(const Dual& a) {
  Dual r(-a.v);
  for (int i = 0; i < ND; ++i) r.d[i] = -a.d[i];
  return r;
}
inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r(a.v * b.v);
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  double ib = 1.0 / b.v;
  for (int i = 0; i < ND; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
inline Dual sqrt(const Dual& a) {
  Dual r(std::sqrt(a.v));
  double s = 0.5 / r.v;
  for (int i = 0; i < ND; ++i) r.d[i] = a.d[i] * s;
  return r;
}
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
using std::sqrt;

// --------------------------------------------------------------------------
// Lens model (Table S1 columns).  Table row layout (12 doubles):
//   type (0 refractive, 1 stop), radius, thickness to next, nd, Vd,
//   semi-diameter, conic, a4, a6, a8, a10, a12
// The material is that of the gap after the surface; nd == 1 is air.
// --------------------------------------------------------------------------
enum { T_REFR = 0, T_STOP = 1 };
constexpr int NCOL = 12;
constexpr int NPAR_SURF = 8;  // c, k, a4..a12, t  (parameter ids s*8 + j)

template <class T>
struct Surf {
  int type;
  T c, k, a[5], t;
  double sd;     // clear semi-diameter (mm)
  double A, B;   // Cauchy coefficients of the medium after (B in um^2)
};

// Two-term Cauchy fit n = A + B / lambda^2 through nd (d line) with the
// F-C dispersion (nd - 1) / Vd (reading: the paper gives glasses as nd/Vd).
void cauchy_from_abbe(double nd, double vd, double* A, double* B) {
  if (vd <= 0.0 || nd == 1.0) {
    *A = nd;
    *B = 0.0;
    return;
  }
  const double lF = 0.4861327, lC = 0.6562725, ld = 0.5875618;  // um
  *B = (nd - 1.0) / vd / (1.0 / (lF * lF) - 1.0 / (lC * lC));
  *A = nd - *B / (ld * ld);
}

inline double index_at(double A, double B, double lam_um) {
  return A + B / (lam_um * lam_um);
}

template <class T>
std::vector<Surf<T>> make_lens(const double* tab, int n) {
  std::vector<Surf<T>> L(n);
  for (int i = 0; i < n; ++i) {
    const double* r = tab + i * NCOL;
    Surf<T>& s = L[i];
    s.type = (int)r[0];
    s.c = (r[1] == 0.0) ? 0.0 : 1.0 / r[1];
    s.t = r[2];
    cauchy_from_abbe(r[3], r[4], &s.A, &s.B);
    s.sd = r[5];
    s.k = r[6];
    for (int j = 0; j < 5; ++j) s.a[j] = r[7 + j];
  }
  return L;
}

// --------------------------------------------------------------------------
// Paraxial optics (first-order y-nu trace), FP64.
// Ray state: height y and slope u in the current medium; refraction at a
// surface of curvature c between indices n1 -> n2:  n2 u2 = n1 u1 - y (n2-n1) c
// --------------------------------------------------------------------------
struct YU {
  double y, u, n;
};

// Trace a paraxial ray given at the vertex plane of surface `from` (before
// refraction there) through surfaces [from, to), ending at the vertex plane
// of surface `to` (before refraction there).  Indices before `from` are
// taken from the table.
YU parax_trace(const std::vector<Surf<double>>& L, double lam_um, double y,
               double u, int from, int to) {
  double n = 1.0;
  if (from > 0) n = index_at(L[from - 1].A, L[from - 1].B, lam_um);
  for (int s = from; s < to; ++s) {
    double n2 = index_at(L[s].A, L[s].B, lam_um);
    if (L[s].type == T_REFR) u = (n * u - y * (n2 - n) * L[s].c) / n2;
    n = n2;
    y = y + L[s].t * u;
  }
  return {y, u, n};
}

struct Parax {
  double efl, bfl;      // at lam
  double z_ep, r_ep;    // entrance pupil (vertex plane of surface 0 is z=0)
  double img_dist;      // paraxial image distance after the last vertex
  double m_sensor;      // chief-ray height at the sensor per unit object height
  double z_sensor;      // sensor plane z
};

int stop_index(const std::vector<Surf<double>>& L) {
  for (size_t i = 0; i < L.size(); ++i)
    if (L[i].type == T_STOP) return (int)i;
  return -1;
}

// Entrance pupil: paraxial image of the stop in object space.  For a ray
// entering at the z=0 plane with height y0 and slope u0, the height at the
// stop plane is M11 y0 + M12 u0; the EP plane is where the chief ray
// (stop-centre ray) crosses the axis in object space.
void entrance_pupil(const std::vector<Surf<double>>& L, double lam_um,
                    double* z_ep, double* r_ep) {
  int s = stop_index(L);
  YU a = parax_trace(L, lam_um, 1.0, 0.0, 0, s);
  YU b = parax_trace(L, lam_um, 0.0, 1.0, 0, s);
  double M11 = a.y, M12 = b.y;
  *z_ep = M12 / M11;
  *r_ep = std::fabs(L[s].sd / M11);
}

// Last surface's vertex z (sum of thicknesses before it).
double z_last_vertex(const std::vector<Surf<double>>& L) {
  double z = 0;
  for (size_t i = 0; i + 1 < L.size(); ++i) z += L[i].t;
  return z;
}

// Image distance after the last vertex for an axial object at depth d (mm
// in front of the z=0 plane).
double image_distance(const std::vector<Surf<double>>& L, double lam_um,
                      double d) {
  YU r = parax_trace(L, lam_um, 1.0, 1.0 / d, 0, (int)L.size() - 1);
  // refraction at the last surface, then the crossing distance
  const Surf<double>& s = L.back();
  double n2 = index_at(s.A, s.B, lam_um);
  double u = r.u;
  if (s.type == T_REFR) u = (r.n * r.u - r.y * (n2 - r.n) * s.c) / n2;
  return -r.y / u;
}

Parax paraxial(const std::vector<Surf<double>>& L, double lam_um, double d) {
  Parax P{};
  // focal length: collimated ray of unit height through all surfaces
  {
    YU r = parax_trace(L, lam_um, 1.0, 0.0, 0, (int)L.size() - 1);
    const Surf<double>& s = L.back();
    double n2 = index_at(s.A, s.B, lam_um);
    double u = r.u;
    if (s.type == T_REFR) u = (r.n * r.u - r.y * (n2 - r.n) * s.c) / n2;
    P.efl = -1.0 / (n2 * u);
    P.bfl = -r.y / u;
  }
  entrance_pupil(L, lam_um, &P.z_ep, &P.r_ep);
  P.img_dist = image_distance(L, lam_um, d);
  // chief ray from unit object height at z=-d through the EP centre
  {
    double u0 = -1.0 / (P.z_ep + d);
    double y0 = 1.0 + u0 * d;
    YU r = parax_trace(L, lam_um, y0, u0, 0, (int)L.size());
    P.m_sensor = r.y;  // parax_trace already transferred by the last thickness
  }
  P.z_sensor = z_last_vertex(L) + L.back().t;
  return P;
}

// Sets the last thickness (sensor distance) so that an axial object at
// focus_mm is in paraxial focus at lam (d line by default).
void focus_lens(std::vector<Surf<double>>& L, double focus_mm) {
  if (focus_mm > 0) L.back().t = image_distance(L, 0.5875618, focus_mm);
}

// --------------------------------------------------------------------------
// Real ray trace (Sec. 3.1).  Coordinates in mm; z along the axis toward the
// sensor; surface 0's vertex at z = 0; radius > 0 puts the centre of
// curvature at +z.
// --------------------------------------------------------------------------
enum RayState {
  R_OK = 0,        // reached the sensor plane
  R_MISS = 1,      // no intersection with a surface
  R_CLIP = 2,      // outside a clear aperture (incl. the stop)
  R_TIR = 3,       // total internal reflection
  R_NEWTON = 4,    // asphere intersection did not converge
  R_BACK = 5,      // travelling away from the sensor
};

template <class T>
struct Ray {
  T x, y, z, dx, dy, dz;
};

template <class T>
struct Hit {
  T x, y, dx, dy, dz;  // sensor landing point and direction
  int state;
  int surf;            // surface where the ray died (-1 if it reached)
  double ap_margin;    // min over surfaces of (semi-diameter - rho), mm
};

template <class T>
bool has_asphere(const Surf<T>& s) {
  for (int j = 0; j < 5; ++j)
    if (val(s.a[j]) != 0.0) return true;
  return false;
}

// Sag z(u) with u = rho^2 and its derivative dz/du (even asphere, Table S1):
//   z = c u / (1 + sqrt(1 - (1+k) c^2 u)) + a4 u^2 + a6 u^3 + ... + a12 u^6
template <class T>
bool sag(const Surf<T>& s, const T& u, T* z, T* dzdu) {
  T arg = T(1.0) - (T(1.0) + s.k) * s.c * s.c * u;
  if (val(arg) < 0.0) return false;
  T q = sqrt(arg);
  T zz = s.c * u / (T(1.0) + q);
  T dz = (val(q) > 0.0) ? s.c / (T(2.0) * q) : T(0.0);
  T up = u;  // u^(m-1) for term m = 2..6
  for (int j = 0; j < 5; ++j) {
    int m = j + 2;
    dz = dz + T((double)m) * s.a[j] * up;
    up = up * u;
    zz = zz + s.a[j] * up;
  }
  *z = zz;
  *dzdu = dz;
  return true;
}

// Intersection parameter along the ray (vertex-local origin o, unit dir d).
// Conic part in closed form (cancellation-free root of
// A t^2 - 2 B t + C = 0 with A = c(dx^2+dy^2+(1+k)dz^2),
// B = dz - c(ox dx + oy dy + (1+k) oz dz), C = c(ox^2+oy^2+(1+k)oz^2) - 2 oz,
// t = C / (B + sqrt(B^2 - A C))); aspheres refine it by Newton on
// F(t) = oz + t dz - sag(rho(t)^2) to |dt| < 1e-12 mm (50 iterations max).
template <class T>
int intersect(const Surf<T>& s, const T& ox, const T& oy, const T& oz,
              const T& dx, const T& dy, const T& dz, T* tout) {
  T t;
  if (s.type == T_STOP || val(s.c) == 0.0) {
    if (val(dz) <= 0.0) return R_BACK;
    t = -oz / dz;
  } else {
    T kk = T(1.0) + s.k;
    T A = s.c * (dx * dx + dy * dy + kk * dz * dz);
    T B = dz - s.c * (ox * dx + oy * dy + kk * oz * dz);
    T C = s.c * (ox * ox + oy * oy + kk * oz * oz) - T(2.0) * oz;
    T disc = B * B - A * C;
    if (val(disc) < 0.0) return R_MISS;
    T den = B + sqrt(disc);
    if (val(den) <= 0.0) return R_MISS;
    t = C / den;
  }
  if (s.type == T_REFR && has_asphere(s)) {
    bool conv = false;
    for (int it = 0; it < 50; ++it) {
      T px = ox + t * dx, py = oy + t * dy;
      T u = px * px + py * py;
      T z, dzdu;
      if (!sag(s, u, &z, &dzdu)) return R_NEWTON;
      T F = oz + t * dz - z;
      T dF = dz - dzdu * T(2.0) * (px * dx + py * dy);
      T step = F / dF;
      t = t - step;
      if (std::fabs(val(step)) < 1e-12) {
        conv = true;
        break;
      }
    }
    if (!conv) return R_NEWTON;
    // one more step so that dual parts equal the implicit derivative
    T px = ox + t * dx, py = oy + t * dy;
    T u = px * px + py * py;
    T z, dzdu;
    if (!sag(s, u, &z, &dzdu)) return R_NEWTON;
    T F = oz + t * dz - z;
    T dF = dz - dzdu * T(2.0) * (px * dx + py * dy);
    t = t - F / dF;
  }
  *tout = t;
  return R_OK;
}

// Sequential trace through all surfaces to the sensor plane.
template <class T>
Hit<T> trace_ray(const std::vector<Surf<T>>& L, double lam_um, Ray<T> r) {
  Hit<T> h{};
  h.state = R_OK;
  h.surf = -1;
  h.ap_margin = 1e300;
  T zv = 0.0;  // vertex z of the current surface
  double n1 = 1.0;
  for (size_t i = 0; i < L.size(); ++i) {
    const Surf<T>& s = L[i];
    T ox = r.x, oy = r.y, oz = r.z - zv;
    T t;
    int st = intersect(s, ox, oy, oz, r.dx, r.dy, r.dz, &t);
    if (st != R_OK) {
      h.state = st;
      h.surf = (int)i;
      return h;
    }
    T px = ox + t * r.dx, py = oy + t * r.dy, pz = oz + t * r.dz;
    double rho = std::sqrt(val(px) * val(px) + val(py) * val(py));
    h.ap_margin = std::min(h.ap_margin, s.sd - rho);
    if (rho > s.sd) {
      h.state = R_CLIP;
      h.surf = (int)i;
      return h;
    }
    r.x = px;
    r.y = py;
    r.z = pz + zv;
    double n2 = index_at(s.A, s.B, lam_um);
    if (s.type == T_REFR) {
      // unit normal from the sag gradient of G = z - sag(x^2 + y^2)
      T u = px * px + py * py, z, dzdu;
      if (!sag(s, u, &z, &dzdu)) {
        h.state = R_MISS;
        h.surf = (int)i;
        return h;
      }
      T gx = T(-2.0) * px * dzdu, gy = T(-2.0) * py * dzdu, gz = T(1.0);
      T gn = sqrt(gx * gx + gy * gy + gz * gz);
      gx = gx / gn;
      gy = gy / gn;
      gz = gz / gn;
      // vector Snell's law, normal oriented along the propagation
      T cosi = gx * r.dx + gy * r.dy + gz * r.dz;
      T eta = T(n1 / n2);
      T k2 = T(1.0) - eta * eta * (T(1.0) - cosi * cosi);
      if (val(k2) < 0.0) {
        h.state = R_TIR;
        h.surf = (int)i;
        return h;
      }
      T g = sqrt(k2) - eta * cosi;
      r.dx = eta * r.dx + g * gx;
      r.dy = eta * r.dy + g * gy;
      r.dz = eta * r.dz + g * gz;
    }
    n1 = n2;
    zv = zv + s.t;
  }
  // zv is now the sensor plane z
  if (val(r.dz) <= 0.0) {
    h.state = R_BACK;
    h.surf = (int)L.size();
    return h;
  }
  T t = (zv - r.z) / r.dz;
  h.x = r.x + t * r.dx;
  h.y = r.y + t * r.dy;
  h.dx = r.dx;
  h.dy = r.dy;
  h.dz = r.dz;
  return h;
}

// --------------------------------------------------------------------------
// Ray set A for one object point (Sec. 3.1): N x N cell-centred samples on
// the entrance-pupil square, kept when inside the pupil disc (exact integer
// test (2i+1-N)^2 + (2j+1-N)^2 <= N^2), each ray on the line from p through
// its sample, started on the EP plane (or 1 mm in front of the first surface
// when the EP lies behind it).
// --------------------------------------------------------------------------
struct Request {
  double h_mm, depth_mm, lam_nm;
  int n_grid, ks;
  double v_mm;  // image height along y (0 for field points on the +x axis)
};

// columns of one request row: h_mm, depth_mm, lambda_nm, n_grid, ks, v_mm
constexpr int REQ_COLS = 6;

struct Sensor {
  double ps, h, f, w, r;  // pixel pitch and DP structure (Eq. S1), all mm
};

struct RayGen {
  double xo, yo, z_ep, r_ep, z_start;
  double xc, yc;  // patch centre on the sensor
};

double front_z(const std::vector<Surf<double>>& L) {
  const Surf<double>& s = L[0];
  double z = 0.0;
  if (s.type == T_REFR) {
    double zz, dd;
    if (sag(s, s.sd * s.sd, &zz, &dd)) z = std::min(0.0, zz);
  }
  return z;
}

RayGen ray_gen_setup(const std::vector<Surf<double>>& L, const Request& q) {
  double lam_um = q.lam_nm * 1e-3;
  Parax P = paraxial(L, lam_um, q.depth_mm);
  RayGen g{};
  // reading: object point from the paraxial chief ray landing at (h, v) on
  // the sensor plane, so that the patch is centred on that landing point
  // (the lens is rotationally symmetric: both coordinates scale by the same
  // chief-ray magnification).
  g.xo = q.h_mm / P.m_sensor;
  g.yo = q.v_mm / P.m_sensor;
  g.z_ep = P.z_ep;
  g.r_ep = P.r_ep;
  double zf = front_z(L);
  g.z_start = (P.z_ep <= zf) ? P.z_ep : zf - 1.0;
  g.xc = q.h_mm;
  g.yc = q.v_mm;
  return g;
}

template <class T>
Ray<T> make_ray(const RayGen& g, const Request& q, int ix, int iy) {
  int N = q.n_grid;
  double ex = (double)(2 * ix + 1 - N) / N * g.r_ep;
  double ey = (double)(2 * iy + 1 - N) / N * g.r_ep;
  double px = g.xo, py = g.yo, pz = -q.depth_mm;
  double vx = ex - px, vy = ey - py, vz = g.z_ep - pz;
  double nv = std::sqrt(vx * vx + vy * vy + vz * vz);
  Ray<T> r;
  if (g.z_start == g.z_ep) {
    r.x = ex;
    r.y = ey;
    r.z = g.z_ep;
  } else {
    double s = (g.z_start - pz) / vz;
    r.x = px + s * vx;
    r.y = py + s * vy;
    r.z = g.z_start;
  }
  r.dx = vx / nv;
  r.dy = vy / nv;
  r.dz = vz / nv;
  return r;
}

inline bool in_pupil(int ix, int iy, int N) {
  long a = 2L * ix + 1 - N, b = 2L * iy + 1 - N;
  return a * a + b * b <= (long)N * N;
}

// --------------------------------------------------------------------------
// DP sub-pixel decision (Eq. 1 / Eq. 2).  For a landing point at offset
// (dxp, dyp) from its pixel centre with tan(theta) = D_x / D_z:
//   inside the microlens disc (radius r):  s = dxp (f - h) / f + h tan(theta)
//   outside:                               s = dxp + h tan(theta)
// and the ray enters L when 0 <= s < w, R when -w <= s < 0, else it is
// missed.  s >= 0 is x >= x_M, s < w is x < x_L and s >= -w is x >= x_R for
// the boundary lines of Eq. (1)/(2), so this is the paper's interval test
// (reading: "L" is the +x sub-pixel; intervals are half-open).
// --------------------------------------------------------------------------
enum Side { S_L = 0, S_R = 1, S_MISS = 2 };

struct Decision {
  int side;
  double margin;  // distance (mm, landing x) to the nearest L/R/miss boundary
};

Decision dp_side(const Sensor& S, double dxp, double dyp, double tan_t) {
  Decision d{};
  double rr = std::sqrt(dxp * dxp + dyp * dyp);
  bool inside = rr <= S.r;
  double sl = inside ? (S.f - S.h) / S.f : 1.0;
  double s = dxp * sl + S.h * tan_t;
  if (s >= 0.0 && s < S.w)
    d.side = S_L;
  else if (s >= -S.w && s < 0.0)
    d.side = S_R;
  else
    d.side = S_MISS;
  double m = std::min({std::fabs(s - S.w), std::fabs(s), std::fabs(s + S.w)}) / sl;
  m = std::min(m, std::fabs(rr - S.r));
  d.margin = m;
  return d;
}

// Per-ray binning record.
struct Bin {
  int state;   // ray state; R_OK rays get side/clipped below
  int side;    // S_L / S_R / S_MISS (valid when state == R_OK)
  int clipped; // landing pixel outside the patch
  int a, b;    // landing pixel (column, row) in patch coordinates
  double fx, fy;  // pixel-centre coordinates of the landing point
  double margin;
};

Bin bin_ray(const Sensor& S, const RayGen& g, int ks, double x, double y,
            double tan_t, int state, double ap_margin) {
  Bin b{};
  b.state = state;
  b.margin = ap_margin;
  if (state != R_OK) return b;
  int p = (ks - 1) / 2;
  b.fx = (x - g.xc) / S.ps + p;
  b.fy = (y - g.yc) / S.ps + p;
  // half-open cell [centre - ps/2, centre + ps/2)
  b.a = (int)std::floor(b.fx + 0.5);
  b.b = (int)std::floor(b.fy + 0.5);
  b.clipped = (b.a < 0 || b.a >= ks || b.b < 0 || b.b >= ks) ? 1 : 0;
  double exm = (0.5 - std::fabs(b.fx - b.a)) * S.ps;
  double eym = (0.5 - std::fabs(b.fy - b.b)) * S.ps;
  double dxp = x - (g.xc + (b.a - p) * S.ps);
  double dyp = y - (g.yc + (b.b - p) * S.ps);
  Decision d = dp_side(S, dxp, dyp, tan_t);
  b.side = d.side;
  b.margin = std::min({b.margin, exm, eym, d.margin});
  return b;
}

// Stats slots per request
enum {
  ST_LAUNCHED = 0, ST_REACHED, ST_L, ST_R, ST_DPMISS, ST_CLIPPED, ST_VIGN,
  ST_OTHER, N_STATS
};

// Traces one request and accumulates Eq. (3) into psf[2][ks][ks]
// (mode 0: unit impulse into the landing pixel; mode 1: unit energy split
// bilinearly over the four nearest pixel centres, L/R from the landing
// pixel, taps outside the patch dropped).
void psf_request(const std::vector<Surf<double>>& L, const Sensor& S,
                 const Request& q, int mode, double* psf, int64_t* st) {
  int ks = q.ks, N = q.n_grid;
  std::fill(psf, psf + 2 * ks * ks, 0.0);
  for (int i = 0; i < N_STATS; ++i) st[i] = 0;
  RayGen g = ray_gen_setup(L, q);
  double lam_um = q.lam_nm * 1e-3;
  for (int iy = 0; iy < N; ++iy)
    for (int ix = 0; ix < N; ++ix) {
      if (!in_pupil(ix, iy, N)) continue;
      st[ST_LAUNCHED]++;
      Ray<double> r = make_ray<double>(g, q, ix, iy);
      Hit<double> h = trace_ray(L, lam_um, r);
      if (h.state != R_OK) {
        st[h.state == R_CLIP ? ST_VIGN : ST_OTHER]++;
        continue;
      }
      st[ST_REACHED]++;
      Bin b = bin_ray(S, g, ks, h.x, h.y, h.dx / h.dz, h.state, h.ap_margin);
      // stats: every reached ray is exactly one of clipped / missed / L / R
      if (b.clipped)
        st[ST_CLIPPED]++;
      else if (b.side == S_MISS)
        st[ST_DPMISS]++;
      else
        st[b.side == S_L ? ST_L : ST_R]++;
      if (b.side == S_MISS) continue;
      double* P = psf + (b.side == S_L ? 0 : ks * ks);
      if (mode == 0) {
        if (b.clipped) continue;
        P[b.b * ks + b.a] += 1.0;
      } else {
        int a0 = (int)std::floor(b.fx), b0 = (int)std::floor(b.fy);
        double wx = b.fx - a0, wy = b.fy - b0;
        for (int jy = 0; jy < 2; ++jy)
          for (int jx = 0; jx < 2; ++jx) {
            int aa = a0 + jx, bb = b0 + jy;
            if (aa < 0 || aa >= ks || bb < 0 || bb >= ks) continue;
            double w = (jx ? wx : 1.0 - wx) * (jy ? wy : 1.0 - wy);
            P[bb * ks + aa] += w;
          }
      }
    }
}

// Sum normalisation (Sec. 3.2): 1 joint (sum L+R = 1), 2 separate (each
// sums to 1), 3 per ray (divide by the number of launched rays), 0 none.
void normalise(double* psf, int ks, int norm, int64_t launched) {
  int n = ks * ks;
  if (norm == 1) {
    double s = 0;
    for (int i = 0; i < 2 * n; ++i) s += psf[i];
    if (s > 0)
      for (int i = 0; i < 2 * n; ++i) psf[i] /= s;
  } else if (norm == 2) {
    for (int side = 0; side < 2; ++side) {
      double s = 0;
      for (int i = 0; i < n; ++i) s += psf[side * n + i];
      if (s > 0)
        for (int i = 0; i < n; ++i) psf[side * n + i] /= s;
    }
  } else if (norm == 3) {
    if (launched > 0)
      for (int i = 0; i < 2 * n; ++i) psf[i] /= (double)launched;
  }
}

std::vector<Surf<double>> load_focused(const double* tab, int n,
                                       double focus_mm) {
  std::vector<Surf<double>> L = make_lens<double>(tab, n);
  focus_lens(L, focus_mm);
  return L;
}

Request req_from(const double* r) {
  Request q;
  q.h_mm = r[0];
  q.depth_mm = r[1];
  q.lam_nm = r[2];
  q.n_grid = (int)r[3];
  q.ks = (int)r[4];
  q.v_mm = r[5];
  return q;
}

Sensor sensor_from(const double* s) { return {s[0], s[1], s[2], s[3], s[4]}; }

template <class F>
void parallel_for(int n, int n_threads, F fn) {
  if (n_threads <= 1 || n <= 1) {
    for (int i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t)
    th.emplace_back([&]() {
      for (;;) {
        int i = next.fetch_add(1);
        if (i >= n) break;
        fn(i);
      }
    });
  for (auto& t : th) t.join();
}

// --------------------------------------------------------------------------
// Gradient of a linear functional of the (bilinear, per-ray normalised) PSF
// bank with respect to lens parameters, by forward-mode dual numbers.
// Ray generation (object point, EP, patch centre) is frozen at the nominal
// lens; only the trace sees the parameters.  Parameter id s*8+j selects
// surface s and j = 0 curvature, 1 conic, 2..6 a4..a12, 7 thickness after
// the surface (the last surface's thickness is the sensor distance).
// --------------------------------------------------------------------------
void seed_param(std::vector<Surf<Dual>>& L, int pid, int slot) {
  int s = pid / NPAR_SURF, j = pid % NPAR_SURF;
  Surf<Dual>& S = L[s];
  Dual* p = (j == 0) ? &S.c : (j == 1) ? &S.k : (j == 7) ? &S.t : &S.a[j - 2];
  p->d[slot] = 1.0;
}

void perturb_param(std::vector<Surf<double>>& L, int pid, double delta) {
  int s = pid / NPAR_SURF, j = pid % NPAR_SURF;
  Surf<double>& S = L[s];
  double* p = (j == 0) ? &S.c : (j == 1) ? &S.k : (j == 7) ? &S.t : &S.a[j - 2];
  *p += delta;
}

std::vector<Surf<Dual>> to_dual(const std::vector<Surf<double>>& L) {
  std::vector<Surf<Dual>> D(L.size());
  for (size_t i = 0; i < L.size(); ++i) {
    const Surf<double>& s = L[i];
    Surf<Dual>& d = D[i];
    d.type = s.type;
    d.c = s.c;
    d.k = s.k;
    d.t = s.t;
    for (int j = 0; j < 5; ++j) d.a[j] = s.a[j];
    d.sd = s.sd;
    d.A = s.A;
    d.B = s.B;
  }
  return D;
}

// Bilinear splat of one ray's weight into the functional G (ks x ks x 2):
// returns sum over taps of G[tap] * weight(tap) * scale.
template <class T>
T splat_functional(const double* G, int ks, int side, const T& fx, const T& fy,
                   int a0, int b0, double scale) {
  T wx = fx - T((double)a0), wy = fy - T((double)b0);
  T acc = 0.0;
  const double* Gs = G + side * ks * ks;
  for (int jy = 0; jy < 2; ++jy)
    for (int jx = 0; jx < 2; ++jx) {
      int aa = a0 + jx, bb = b0 + jy;
      if (aa < 0 || aa >= ks || bb < 0 || bb >= ks) continue;
      T w = (jx ? wx : T(1.0) - wx) * (jy ? wy : T(1.0) - wy);
      acc = acc + T(Gs[bb * ks + aa] * scale) * w;
    }
  return acc;
}

}  // namespace

// ==========================================================================
// C interface (ctypes).  All return 0 on success, negative on bad input.
// ==========================================================================
extern "C" {

// out[8] = efl, bfl, z_ep, r_ep, sensor distance (last thickness),
//          m_sensor(depth), image distance(depth), z_sensor
int or_lens_info(const double* tab, int n, double focus_mm, double lam_nm,
                 double depth_mm, double* out) {
  if (!tab || n < 1 || !out) return -1;
  auto L = load_focused(tab, n, focus_mm);
  if (stop_index(L) < 0) return -2;
  Parax P = paraxial(L, lam_nm * 1e-3, depth_mm);
  out[0] = P.efl;
  out[1] = P.bfl;
  out[2] = P.z_ep;
  out[3] = P.r_ep;
  out[4] = L.back().t;
  out[5] = P.m_sensor;
  out[6] = P.img_dist;
  out[7] = P.z_sensor;
  return 0;
}

// Per-ray record of one request, in pupil raster order (iy major) over the
// in-pupil samples.  out[k*12 + ...] = x, y, dx, dy, dz, state, side,
// clipped, a, b, margin, died-at-surface.  *n_rays = number written.
int or_trace_hits(const double* tab, int n, double focus_mm, const double* req,
                  const double* sensor, double* out, int max_rays,
                  int* n_rays) {
  if (!tab || !req || !sensor || !out || !n_rays) return -1;
  auto L = load_focused(tab, n, focus_mm);
  if (stop_index(L) < 0) return -2;
  Request q = req_from(req);
  Sensor S = sensor_from(sensor);
  RayGen g = ray_gen_setup(L, q);
  double lam_um = q.lam_nm * 1e-3;
  int k = 0, N = q.n_grid;
  for (int iy = 0; iy < N; ++iy)
    for (int ix = 0; ix < N; ++ix) {
      if (!in_pupil(ix, iy, N)) continue;
      if (k >= max_rays) return -3;
      Ray<double> r = make_ray<double>(g, q, ix, iy);
      Hit<double> h = trace_ray(L, lam_um, r);
      double* o = out + (size_t)k * 12;
      for (int j = 0; j < 12; ++j) o[j] = 0;
      o[5] = h.state;
      o[11] = h.surf;
      o[10] = h.ap_margin;
      if (h.state == R_OK) {
        Bin b = bin_ray(S, g, q.ks, h.x, h.y, h.dx / h.dz, h.state, h.ap_margin);
        o[0] = h.x;
        o[1] = h.y;
        o[2] = h.dx;
        o[3] = h.dy;
        o[4] = h.dz;
        o[6] = b.side;
        o[7] = b.clipped;
        o[8] = b.a;
        o[9] = b.b;
        o[10] = b.margin;
      }
      ++k;
    }
  *n_rays = k;
  return 0;
}

// PSF bank: reqs[i*REQ_COLS..] = h_mm, depth_mm, lambda_nm, n_grid, ks, v_mm; the PSFs are
// written back to back ([2][ks][ks] each, in request order).  stats[i*8..]
// = launched, reached, L, R, DP-missed, clipped, vignetted, other.
int or_psf_bank(const double* tab, int n, double focus_mm, const double* reqs,
                int n_req, const double* sensor, int mode, int norm,
                double* bank, int64_t* stats, int n_threads) {
  if (!tab || !reqs || !sensor || !bank || !stats || n_req < 0) return -1;
  auto L = load_focused(tab, n, focus_mm);
  if (stop_index(L) < 0) return -2;
  Sensor S = sensor_from(sensor);
  std::vector<size_t> off(n_req + 1, 0);
  for (int i = 0; i < n_req; ++i) {
    int ks = (int)reqs[i * REQ_COLS + 4];
    if (ks < 1 || ks % 2 == 0) return -4;
    off[i + 1] = off[i] + 2 * (size_t)ks * ks;
  }
  parallel_for(n_req, n_threads, [&](int i) {
    Request q = req_from(reqs + i * REQ_COLS);
    psf_request(L, S, q, mode, bank + off[i], stats + i * N_STATS);
    normalise(bank + off[i], q.ks, norm, stats[i * N_STATS + ST_LAUNCHED]);
  });
  return 0;
}

// Value of the functional  sum_i sum_taps G_i[tap] * PSF_i[tap]  for the
// bilinear PSFs scaled by 1/launched, with parameter perturbations delta
// (param ids pids) applied to the traced lens; ray generation stays at the
// nominal lens.  freeze != 0 keeps every ray's discrete decisions (state,
// side, splat base pixel) at their nominal values.
int or_trace_functional(const double* tab, int n, double focus_mm,
                        const double* reqs, int n_req, const double* sensor,
                        const double* G, const int* pids, const double* delta,
                        int n_par, int freeze, double* out) {
  if (!tab || !reqs || !sensor || !G || !out) return -1;
  auto L0 = load_focused(tab, n, focus_mm);
  if (stop_index(L0) < 0) return -2;
  auto L1 = L0;
  for (int j = 0; j < n_par; ++j) perturb_param(L1, pids[j], delta[j]);
  Sensor S = sensor_from(sensor);
  double total = 0.0;
  size_t goff = 0;
  for (int i = 0; i < n_req; ++i) {
    Request q = req_from(reqs + i * REQ_COLS);
    RayGen g = ray_gen_setup(L0, q);
    double lam_um = q.lam_nm * 1e-3;
    int N = q.n_grid, ks = q.ks;
    int64_t launched = 0;
    for (int iy = 0; iy < N; ++iy)
      for (int ix = 0; ix < N; ++ix) launched += in_pupil(ix, iy, N);
    double scale = launched ? 1.0 / launched : 0.0;
    for (int iy = 0; iy < N; ++iy)
      for (int ix = 0; ix < N; ++ix) {
        if (!in_pupil(ix, iy, N)) continue;
        Ray<double> r = make_ray<double>(g, q, ix, iy);
        Hit<double> h0 = trace_ray(L0, lam_um, r);
        Hit<double> h1 = trace_ray(L1, lam_um, r);
        Hit<double>& hd = freeze ? h0 : h1;
        if (hd.state != R_OK || h1.state != R_OK) continue;
        Bin bd = bin_ray(S, g, ks, hd.x, hd.y, hd.dx / hd.dz, hd.state, 0);
        if (bd.side == S_MISS) continue;
        int p = (ks - 1) / 2;
        double fx = (h1.x - g.xc) / S.ps + p, fy = (h1.y - g.yc) / S.ps + p;
        int a0 = (int)std::floor(bd.fx), b0 = (int)std::floor(bd.fy);
        if (!freeze) {
          a0 = (int)std::floor(fx);
          b0 = (int)std::floor(fy);
        }
        total += splat_functional<double>(G + goff, ks, bd.side, fx, fy, a0, b0,
                                          scale);
      }
    goff += 2 * (size_t)ks * ks;
  }
  *out = total;
  return 0;
}

// Gradient of the functional above at delta = 0 with respect to the n_par
// (<= 24) parameters pids, by dual numbers.  grads[n_par].
int or_trace_grad(const double* tab, int n, double focus_mm, const double* reqs,
                  int n_req, const double* sensor, const double* G,
                  const int* pids, int n_par, double* grads, int n_threads) {
  if (!tab || !reqs || !sensor || !G || !grads || n_par > ND) return -1;
  auto L0 = load_focused(tab, n, focus_mm);
  if (stop_index(L0) < 0) return -2;
  for (int j = 0; j < n_par; ++j)
    if (pids[j] < 0 || pids[j] / NPAR_SURF >= n) return -4;
  auto LD = to_dual(L0);
  for (int j = 0; j < n_par; ++j) seed_param(LD, pids[j], j);
  Sensor S = sensor_from(sensor);
  std::vector<size_t> goff(n_req + 1, 0);
  for (int i = 0; i < n_req; ++i) {
    int ks = (int)reqs[i * REQ_COLS + 4];
    goff[i + 1] = goff[i] + 2 * (size_t)ks * ks;
  }
  std::vector<double> part((size_t)n_req * ND, 0.0);
  parallel_for(n_req, n_threads, [&](int i) {
    Request q = req_from(reqs + i * REQ_COLS);
    RayGen g = ray_gen_setup(L0, q);
    double lam_um = q.lam_nm * 1e-3;
    int N = q.n_grid, ks = q.ks, p = (ks - 1) / 2;
    int64_t launched = 0;
    for (int iy = 0; iy < N; ++iy)
      for (int ix = 0; ix < N; ++ix) launched += in_pupil(ix, iy, N);
    double scale = launched ? 1.0 / launched : 0.0;
    Dual acc = 0.0;
    for (int iy = 0; iy < N; ++iy)
      for (int ix = 0; ix < N; ++ix) {
        if (!in_pupil(ix, iy, N)) continue;
        Ray<Dual> r = make_ray<Dual>(g, q, ix, iy);
        Hit<Dual> h = trace_ray(LD, lam_um, r);
        if (h.state != R_OK) continue;
        Bin b = bin_ray(S, g, ks, h.x.v, h.y.v, h.dx.v / h.dz.v, h.state, 0);
        if (b.side == S_MISS) continue;
        Dual fx = (h.x - Dual(g.xc)) / Dual(S.ps) + Dual((double)p);
        Dual fy = (h.y - Dual(g.yc)) / Dual(S.ps) + Dual((double)p);
        int a0 = (int)std::floor(b.fx), b0 = (int)std::floor(b.fy);
        acc = acc + splat_functional<Dual>(G + goff[i], ks, b.side, fx, fy, a0,
                                           b0, scale);
      }
    for (int j = 0; j < ND; ++j) part[(size_t)i * ND + j] = acc.d[j];
  });
  for (int j = 0; j < n_par; ++j) {
    double s = 0;
    for (int i = 0; i < n_req; ++i) s += part[(size_t)i * ND + j];
    grads[j] = s;
  }
  return 0;
}

// --------------------------------------------------------------------------
// Rendering (supplement, "Local DP PSF convolution"): for each output pixel
// (y, x) with its own kernels K_L, K_R (ks x ks, p = (ks-1)/2),
//   out_L[n, c, y, x] = sum_{i,j} Ipad[n, c, y+i, x+j] * K_L[ks-1-i][ks-1-j]
// where Ipad is the input replicate-padded by p; likewise R; output channels
// are [L(c = 0..C-1), R(c = 0..C-1)].
//
// Kernel source, bank mode: the pixel's kernel for channel c is
//   (1 - t) * bank[f][z0][lam] + t * bank[f][z0 + 1][lam],
// lam = c when the bank has C wavelengths (else 0), f the field height
// nearest to the pixel's radial image height, and (z0, t) the bracket of the
// pixel depth linear in inverse depth (clamped at both ends).  This selection
// is an integer decision and is taken in FP32 with unfused operations:
//   X = ((float)col - 0.5f*(W-1)) * pitch,  Y likewise with rows,
//   rho = sqrtf(X*X + Y*Y); q = 1.0f / depth; iq_j = 1.0f / depths_j.
// Map mode: psf_map[y][x][2][ks][ks] shared by all channels and images.
// --------------------------------------------------------------------------
namespace {

struct Sel {
  int f, z0, z1;
  double t;
  bool mirror_x, mirror_y;  // quadrant bank: flips of the first-quadrant PSF
};

// Nearest field height to r: bracket i with fh[i] <= r < fh[i+1], then the
// closer end (ties to the lower index); clamped at both ends.
int nearest_height(const float* fh, int F, float r) {
  if (r <= fh[0]) return 0;
  if (r >= fh[F - 1]) return F - 1;
  int i = 0;
  while (i + 1 < F && fh[i + 1] <= r) ++i;
  volatile float dlo = r - fh[i];
  volatile float dhi = fh[i + 1] - r;
  return (dhi < dlo) ? i + 1 : i;
}

// mode 0 (radial bank): f = the height nearest to the radial image height.
// mode 1 (first-quadrant bank [F][F]): f = ix * F + iy with ix, iy the
// heights nearest to |X| and |Y|; a pixel with X < 0 (Y < 0) uses the PSF
// mirrored about the y (x) axis, the flip symmetry of the DP PSF (Sec. 5.3).
Sel select_slice(int row, int col, int H, int W, float pitch, float depth,
                 const float* fh, int F, const float* iq, int Z, int mode = 0) {
  volatile float X = ((float)col - 0.5f * (float)(W - 1)) * pitch;
  volatile float Y = ((float)row - 0.5f * (float)(H - 1)) * pitch;
  Sel s{};
  if (mode == 1) {
    s.f = nearest_height(fh, F, std::fabs((float)X)) * F + nearest_height(fh, F, std::fabs((float)Y));
    s.mirror_x = X < 0.f;
    s.mirror_y = Y < 0.f;
  } else {
    volatile float X2 = X * X;
    volatile float Y2 = Y * Y;
    volatile float R2 = X2 + Y2;
    s.f = nearest_height(fh, F, std::sqrt((float)R2));
  }
  if (Z == 1) {
    s.z0 = s.z1 = 0;
    s.t = 0.0;
    return s;
  }
  volatile float q = 1.0f / depth;
  if (q >= iq[0]) {
    s.z0 = 0;
    s.t = 0.0;
  } else if (q <= iq[Z - 1]) {
    s.z0 = Z - 2;
    s.t = 1.0;
  } else {
    int j = 0;
    while (j + 1 < Z && iq[j + 1] >= q) ++j;  // iq[j] >= q > iq[j+1]
    volatile float num = iq[j] - q;
    volatile float den = iq[j] - iq[j + 1];
    volatile float tf = num / den;
    s.z0 = j;
    s.t = (double)tf;
  }
  s.z1 = s.z0 + 1;
  return s;
}

inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

struct BankDesc {
  const double* bank;
  int F, Z, NL, ks;
  const float* fh;
  const float* iq;
  float pitch;
  int mode;  // 0 radial [F], 1 first quadrant [F][F]
};

// Fills K[2][ks][ks] (unflipped, rows = y, columns = x) for pixel (row, col)
// of image n, channel c.  Quadrant bank: a mirror about the y axis reverses
// the columns and exchanges L and R (the DP split is along x), a mirror
// about the x axis reverses the rows.
void pixel_kernel(const BankDesc& B, int row, int col, int H, int W, float depth,
                  int lam, double* K, Sel* sel_out) {
  Sel s = select_slice(row, col, H, W, B.pitch, depth, B.fh, B.F, B.iq, B.Z, B.mode);
  const int ks = B.ks;
  size_t n1 = (size_t)ks * ks, n2 = 2 * n1;
  const double* k0 = B.bank + (((size_t)s.f * B.Z + s.z0) * B.NL + lam) * n2;
  const double* k1 = B.bank + (((size_t)s.f * B.Z + s.z1) * B.NL + lam) * n2;
  for (int side = 0; side < 2; ++side)
    for (int a = 0; a < ks; ++a)
      for (int b = 0; b < ks; ++b) {
        const int side_src = s.mirror_x ? 1 - side : side;
        const int a_src = s.mirror_y ? ks - 1 - a : a;
        const int b_src = s.mirror_x ? ks - 1 - b : b;
        const size_t src = side_src * n1 + (size_t)a_src * ks + b_src;
        K[side * n1 + (size_t)a * ks + b] = (1.0 - s.t) * k0[src] + s.t * k1[src];
      }
  if (sel_out) *sel_out = s;
}

}  // namespace

// Bank-mode render.  aif (N,C,H,W) f64, depth_m (N,H,W) f32, bank
// [F][Z][NL][2][ks][ks] f64, field_h_mm[F] f32 (ascending), depths_m[Z] f32
// (ascending), out (N,2C,H,W) f64.
// field_mode 0: bank [F][Z][NL][2][ks][ks] over radial heights; 1: bank
// [F][F][Z][NL][2][ks][ks] over the first quadrant (see select_slice).
int or_render_bank_mode(const double* aif, int N, int C, int H, int W,
                        const float* depth_m, const double* bank, int F, int Z,
                        int NL, int ks, const float* field_h_mm,
                        const float* depths_m, float pitch_mm, int field_mode, double* out,
                        int n_threads) {
  if (!aif || !depth_m || !bank || !out || ks < 1 || ks % 2 == 0) return -1;
  if (!(NL == C || NL == 1)) return -4;
  if (field_mode != 0 && field_mode != 1) return -1;
  std::vector<float> iq(Z);
  for (int j = 0; j < Z; ++j) iq[j] = 1.0f / depths_m[j];
  BankDesc B{bank, F, Z, NL, ks, field_h_mm, iq.data(), pitch_mm, field_mode};
  int p = (ks - 1) / 2;
  parallel_for(N * H, n_threads, [&](int nr) {
    int n = nr / H, y = nr % H;
    std::vector<double> K(2 * (size_t)ks * ks);
    for (int x = 0; x < W; ++x)
      for (int c = 0; c < C; ++c) {
        int lam = (NL == C) ? c : 0;
        pixel_kernel(B, y, x, H, W, depth_m[((size_t)n * H + y) * W + x], lam,
                     K.data(), nullptr);
        const double* img = aif + ((size_t)n * C + c) * H * W;
        double accL = 0, accR = 0;
        for (int i = 0; i < ks; ++i)
          for (int j = 0; j < ks; ++j) {
            double v = img[(size_t)clampi(y + i - p, 0, H - 1) * W +
                           clampi(x + j - p, 0, W - 1)];
            int kk = (ks - 1 - i) * ks + (ks - 1 - j);
            accL += v * K[kk];
            accR += v * K[(size_t)ks * ks + kk];
          }
        out[(((size_t)n * 2 * C + c) * H + y) * W + x] = accL;
        out[(((size_t)n * 2 * C + C + c) * H + y) * W + x] = accR;
      }
  });
  return 0;
}

int or_render_bank(const double* aif, int N, int C, int H, int W,
                   const float* depth_m, const double* bank, int F, int Z,
                   int NL, int ks, const float* field_h_mm,
                   const float* depths_m, float pitch_mm, double* out,
                   int n_threads) {
  return or_render_bank_mode(aif, N, C, H, W, depth_m, bank, F, Z, NL, ks, field_h_mm,
                             depths_m, pitch_mm, 0, out, n_threads);
}

// Bank-mode render of selected pixels only: pix[i*3..] = (n, y, x);
// out[i*2C + c] = L of channel c, out[i*2C + C + c] = R.
int or_render_bank_pixels_mode(const double* aif, int N, int C, int H, int W,
                               const float* depth_m, const double* bank, int F, int Z,
                               int NL, int ks, const float* field_h_mm,
                               const float* depths_m, float pitch_mm, int field_mode,
                               const int* pix, int npix, double* out, int n_threads) {
  if (!aif || !depth_m || !bank || !pix || !out || ks < 1 || ks % 2 == 0) return -1;
  if (!(NL == C || NL == 1)) return -4;
  if (field_mode != 0 && field_mode != 1) return -1;
  std::vector<float> iq(Z);
  for (int j = 0; j < Z; ++j) iq[j] = 1.0f / depths_m[j];
  BankDesc B{bank, F, Z, NL, ks, field_h_mm, iq.data(), pitch_mm, field_mode};
  int p = (ks - 1) / 2;
  parallel_for(npix, n_threads, [&](int i) {
    int n = pix[3 * i], y = pix[3 * i + 1], x = pix[3 * i + 2];
    std::vector<double> K(2 * (size_t)ks * ks);
    for (int c = 0; c < C; ++c) {
      int lam = (NL == C) ? c : 0;
      pixel_kernel(B, y, x, H, W, depth_m[((size_t)n * H + y) * W + x], lam, K.data(),
                   nullptr);
      const double* img = aif + ((size_t)n * C + c) * H * W;
      double accL = 0, accR = 0;
      for (int a = 0; a < ks; ++a)
        for (int b = 0; b < ks; ++b) {
          double v = img[(size_t)clampi(y + a - p, 0, H - 1) * W + clampi(x + b - p, 0, W - 1)];
          int kk = (ks - 1 - a) * ks + (ks - 1 - b);
          accL += v * K[kk];
          accR += v * K[(size_t)ks * ks + kk];
        }
      out[(size_t)i * 2 * C + c] = accL;
      out[(size_t)i * 2 * C + C + c] = accR;
    }
  });
  return 0;
}

int or_render_bank_pixels(const double* aif, int N, int C, int H, int W,
                          const float* depth_m, const double* bank, int F, int Z,
                          int NL, int ks, const float* field_h_mm,
                          const float* depths_m, float pitch_mm, const int* pix,
                          int npix, double* out, int n_threads) {
  return or_render_bank_pixels_mode(aif, N, C, H, W, depth_m, bank, F, Z, NL, ks, field_h_mm,
                                    depths_m, pitch_mm, 0, pix, npix, out, n_threads);
}

// Map-mode render: psf_map (H,W,2,ks,ks) f64.
int or_render_map(const double* aif, int N, int C, int H, int W,
                  const double* psf_map, int ks, double* out) {
  if (!aif || !psf_map || !out || ks < 1 || ks % 2 == 0) return -1;
  int p = (ks - 1) / 2;
  size_t n2 = (size_t)ks * ks;
  for (int n = 0; n < N; ++n)
    for (int c = 0; c < C; ++c)
      for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
          const double* K = psf_map + ((size_t)y * W + x) * 2 * n2;
          const double* img = aif + ((size_t)n * C + c) * H * W;
          double accL = 0, accR = 0;
          for (int i = 0; i < ks; ++i)
            for (int j = 0; j < ks; ++j) {
              double v = img[(size_t)clampi(y + i - p, 0, H - 1) * W +
                             clampi(x + j - p, 0, W - 1)];
              size_t kk = (size_t)(ks - 1 - i) * ks + (ks - 1 - j);
              accL += v * K[kk];
              accR += v * K[n2 + kk];
            }
          out[(((size_t)n * 2 * C + c) * H + y) * W + x] = accL;
          out[(((size_t)n * 2 * C + C + c) * H + y) * W + x] = accR;
        }
  return 0;
}

// Adjoint of or_render_bank with respect to the image and the bank:
// grad_aif (N,C,H,W) and grad_bank (same layout as bank) are overwritten.
// Replicate padding is adjoined by accumulating into the clamped source.
int or_render_bank_bwd_mode(const double* grad_out, const double* aif, int N, int C,
                            int H, int W, const float* depth_m, const double* bank,
                            int F, int Z, int NL, int ks, const float* field_h_mm,
                            const float* depths_m, float pitch_mm, int field_mode,
                            double* grad_aif, double* grad_bank) {
  if (!grad_out || !aif || !depth_m || !bank || !grad_aif || !grad_bank)
    return -1;
  if (!(NL == C || NL == 1) || ks < 1 || ks % 2 == 0) return -4;
  if (field_mode != 0 && field_mode != 1) return -1;
  std::vector<float> iq(Z);
  for (int j = 0; j < Z; ++j) iq[j] = 1.0f / depths_m[j];
  BankDesc B{bank, F, Z, NL, ks, field_h_mm, iq.data(), pitch_mm, field_mode};
  const int cells = field_mode == 1 ? F * F : F;
  int p = (ks - 1) / 2;
  size_t n2 = (size_t)ks * ks;
  std::fill(grad_aif, grad_aif + (size_t)N * C * H * W, 0.0);
  std::fill(grad_bank, grad_bank + (size_t)cells * Z * NL * 2 * n2, 0.0);
  std::vector<double> K(2 * n2), dK(2 * n2);
  for (int n = 0; n < N; ++n)
    for (int c = 0; c < C; ++c) {
      int lam = (NL == C) ? c : 0;
      const double* img = aif + ((size_t)n * C + c) * H * W;
      double* gimg = grad_aif + ((size_t)n * C + c) * H * W;
      for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
          Sel s;
          pixel_kernel(B, y, x, H, W, depth_m[((size_t)n * H + y) * W + x], lam,
                       K.data(), &s);
          double gL = grad_out[(((size_t)n * 2 * C + c) * H + y) * W + x];
          double gR = grad_out[(((size_t)n * 2 * C + C + c) * H + y) * W + x];
          for (int i = 0; i < ks; ++i)
            for (int j = 0; j < ks; ++j) {
              size_t src = (size_t)clampi(y + i - p, 0, H - 1) * W +
                           clampi(x + j - p, 0, W - 1);
              size_t kk = (size_t)(ks - 1 - i) * ks + (ks - 1 - j);
              gimg[src] += gL * K[kk] + gR * K[n2 + kk];
              dK[kk] = gL * img[src];
              dK[n2 + kk] = gR * img[src];
            }
          // dK is the gradient of the pixel's kernel; each of its elements
          // is a stored element (mirrored for a quadrant bank's flips)
          double* b0 = grad_bank + (((size_t)s.f * Z + s.z0) * NL + lam) * 2 * n2;
          double* b1 = grad_bank + (((size_t)s.f * Z + s.z1) * NL + lam) * 2 * n2;
          for (int side = 0; side < 2; ++side)
            for (int a = 0; a < ks; ++a)
              for (int b = 0; b < ks; ++b) {
                const int side_src = s.mirror_x ? 1 - side : side;
                const int a_src = s.mirror_y ? ks - 1 - a : a;
                const int b_src = s.mirror_x ? ks - 1 - b : b;
                const size_t src = side_src * n2 + (size_t)a_src * ks + b_src;
                const double g = dK[side * n2 + (size_t)a * ks + b];
                b0[src] += (1.0 - s.t) * g;
                b1[src] += s.t * g;
              }
        }
    }
  return 0;
}

int or_render_bank_bwd(const double* grad_out, const double* aif, int N, int C,
                       int H, int W, const float* depth_m, const double* bank,
                       int F, int Z, int NL, int ks, const float* field_h_mm,
                       const float* depths_m, float pitch_mm, double* grad_aif,
                       double* grad_bank) {
  return or_render_bank_bwd_mode(grad_out, aif, N, C, H, W, depth_m, bank, F, Z, NL, ks,
                                 field_h_mm, depths_m, pitch_mm, 0, grad_aif, grad_bank);
}

// Per-pixel bank selection as the renderer takes it (for tests):
// out[(y*W+x)*4 ..] = f, z0, z1, t.
int or_render_select(int H, int W, const float* depth_m, const float* field_h_mm,
                     int F, const float* depths_m, int Z, float pitch_mm,
                     double* out) {
  std::vector<float> iq(Z);
  for (int j = 0; j < Z; ++j) iq[j] = 1.0f / depths_m[j];
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      Sel s = select_slice(y, x, H, W, pitch_mm, depth_m[(size_t)y * W + x],
                           field_h_mm, F, iq.data(), Z);
      double* o = out + ((size_t)y * W + x) * 4;
      o[0] = s.f;
      o[1] = s.z0;
      o[2] = s.z1;
      o[3] = s.t;
    }
  return 0;
}

}  // extern "C"
