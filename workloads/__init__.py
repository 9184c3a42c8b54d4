"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module only *describes* inputs: lens prescriptions, DP pixel constants,
PSF request grids and synthetic scenes (all-in-focus images and depth maps).
It performs none of the simulator's arithmetic (no paraxial optics, no ray
tracing, no binning, no rendering).  Everything is deterministic for a given
seed (numpy PCG64).

Lens tables are float64 arrays of shape (n_surfaces, 12) with the columns of
the paper's lens tables (Table S1/S2): surface type, radius, thickness to the
next surface, material after the surface as (nd, Vd), clear semi-diameter,
conic and the even-asphere coefficients a4..a12.  The last row's thickness is
the distance from the last surface to the sensor plane; callers may override
it with a focus distance.
"""
from __future__ import annotations

import math
import numpy as np

# column indices of a lens table
COL_TYPE, COL_R, COL_T, COL_ND, COL_VD, COL_SD, COL_K = 0, 1, 2, 3, 4, 5, 6
COL_A4 = 7  # a4, a6, a8, a10, a12 occupy columns 7..11
N_COLS = 12
SURF_REFRACT, SURF_STOP = 0, 1

# Dual-pixel structure constants as multiples of the pixel pitch (Eq. S1).
DP_H, DP_F, DP_W, DP_R = 0.78, 1.44, 0.30, 0.50

# Fraunhofer lines used by the configurations (nm): C, d, F.
LAMBDA_C, LAMBDA_D, LAMBDA_F = 656.2725, 587.5618, 486.1327
# channel c of an RGB image is traced at this wavelength (R, G, B)
RGB_LAMBDAS_NM = (LAMBDA_C, LAMBDA_D, LAMBDA_F)

CROWN = (1.5168, 64.17)   # N-BK7-like
FLINT = (1.62004, 36.37)  # F2-like
AIR = (1.0, 0.0)


def _row(kind, radius, thick, glass, semi, conic=0.0, asph=(0, 0, 0, 0, 0)):
    r = np.zeros(N_COLS)
    r[COL_TYPE] = kind
    r[COL_R] = radius
    r[COL_T] = thick
    r[COL_ND], r[COL_VD] = glass
    r[COL_SD] = semi
    r[COL_K] = conic
    r[COL_A4:COL_A4 + 5] = asph
    return r


def singlet_f2() -> np.ndarray:
    """Biconvex N-BK7 singlet, R1 = +51.68 mm, R2 = -51.68 mm, 5 mm thick,
    stop (12.5 mm radius) in the vertex plane of the first surface, n = 1.5168
    (non-dispersive).  The last thickness is a placeholder: callers focus it."""
    return np.stack([
        _row(SURF_STOP, 0.0, 0.0, AIR, 12.5),
        _row(SURF_REFRACT, 51.68, 5.0, (1.5168, 0.0), 14.0),
        _row(SURF_REFRACT, -51.68, 50.0, AIR, 14.0),
    ])


def doublet_pair_f18(seed: int = 236) -> np.ndarray:
    """Six-surface f ~ 24 mm, f/1.8 lens: two cemented crown/flint doublets.

    The outer surfaces S1 and S6 are even aspheres whose conic is drawn from
    U[-1, 0] and whose a4..a10 have magnitudes 1e-5, 1e-7, 1e-9, 1e-12 with a
    random sign (seeded).  The stop (radius 24/3.6 mm) sits in the vertex
    plane of S1.  Radii were scaled so that the paraxial EFL at 587.6 nm is
    24.0 mm.  The default seed was picked among 0..299 as the draw with the
    smallest on-axis RMS spot at 1 m (5.4 um): the draw ranges alone allow
    lenses whose in-focus blur exceeds a 65 px patch.
    """
    rng = np.random.default_rng(seed)
    s = 0.6435436280753327
    R = [30 * s, -25 * s, -80 * s, 40 * s, -30 * s, 200 * s]
    mags = np.array([1e-5, 1e-7, 1e-9, 1e-12])

    def asph():
        a = mags * rng.choice([-1.0, 1.0], size=4)
        return (a[0], a[1], a[2], a[3], 0.0)

    k1 = -rng.uniform(0.0, 1.0)
    a1 = asph()
    k6 = -rng.uniform(0.0, 1.0)
    a6 = asph()
    sd = 8.0
    return np.stack([
        _row(SURF_STOP, 0.0, 0.0, AIR, 24.0 / 3.6),
        _row(SURF_REFRACT, R[0], 4.0, CROWN, sd, k1, a1),
        _row(SURF_REFRACT, R[1], 1.5, FLINT, sd),
        _row(SURF_REFRACT, R[2], 1.5, AIR, sd),
        _row(SURF_REFRACT, R[3], 3.5, CROWN, sd),
        _row(SURF_REFRACT, R[4], 1.5, FLINT, sd),
        _row(SURF_REFRACT, R[5], 17.0, AIR, sd, k6, a6),
    ])


def spherical4(seed: int = 11) -> np.ndarray:
    """Four-surface all-spherical lens (two air-spaced singlets), radii drawn
    within +-10 % of (40, -60, 30, -100) mm, stop radius 6 mm in front."""
    rng = np.random.default_rng(seed)
    base = np.array([40.0, -60.0, 30.0, -100.0])
    R = base * rng.uniform(0.9, 1.1, size=4)
    sd = 9.0
    return np.stack([
        _row(SURF_STOP, 0.0, 0.0, AIR, 6.0),
        _row(SURF_REFRACT, R[0], 4.0, CROWN, sd),
        _row(SURF_REFRACT, R[1], 2.0, AIR, sd),
        _row(SURF_REFRACT, R[2], 3.5, FLINT if rng.uniform() < 0.5 else CROWN, sd),
        _row(SURF_REFRACT, R[3], 30.0, AIR, sd),
    ])


def canon_rf50() -> np.ndarray:
    """Canon RF50mm F/1.8 prescription as printed in Table S1 (aperture row =
    stop; material is that of the gap after the surface; diameter -> semi)."""
    rows = [
        (28.621, 4.20, (1.83481, 42.7), 29.99, None),
        (68.136, 0.18, AIR, 28.48, None),
        (17.772, 6.70, (1.79952, 42.2), 23.90, None),
        (59.525, 1.10, (1.80518, 25.4), 20.78, None),
        (11.427, 5.27, AIR, 16.78, None),
        ("stop", 6.20, AIR, 16.24, None),
        (-16.726, 0.90, (1.67270, 32.1), 14.95, None),
        (-29.829, 0.83, AIR, 15.46, None),
        (-25.000, 2.95, (1.53110, 55.9), 15.52,
         (-4.12032e-05, -2.90015e-07, -4.67119e-09, 7.90646e-11, -9.28470e-13)),
        (-18.373, 0.98, AIR, 18.14,
         (-2.41619e-05, -3.29146e-07, 1.91098e-10, -9.28593e-13, -2.29193e-13)),
        (280.004, 4.60, (1.73400, 51.5), 24.43, None),
        (-34.002, 25.67, AIR, 25.71, None),
    ]
    return _table(rows)


def canon_rf35() -> np.ndarray:
    """Canon RF35mm F/1.8 prescription as printed in Table S2."""
    rows = [
        (800.000, 1.00, (1.80810, 22.8), 27.80, None),
        (33.296, 1.92, AIR, 25.64, None),
        (103.801, 3.11, (2.00100, 29.1), 25.57, None),
        (-86.901, 4.09, AIR, 25.07, None),
        (-47.674, 1.30, (1.51742, 52.4), 20.44, None),
        (17.367, 5.73, (1.90043, 37.4), 21.60, None),
        (777.674, 3.72, AIR, 21.26, None),
        ("stop", 3.62, AIR, 20.16, None),
        (64.497, 2.12, (1.69680, 55.5), 19.04, None),
        (-262.934, 3.56, AIR, 18.69, None),
        (-35.963, 1.30, (1.58313, 59.4), 17.10,
         (-4.61997e-05, -9.22837e-08, -4.60687e-10, 1.65555e-13, 0.0)),
        (-93.550, 0.13, AIR, 17.19, None),
        (-84.988, 6.26, (1.88300, 40.8), 17.29, None),
        (-12.701, 1.00, (1.85478, 24.8), 18.97, None),
        (135.000, 5.27, AIR, 22.77, None),
        (800.000, 7.35, (1.90043, 37.4), 31.72, None),
        (-28.799, 0.95, AIR, 33.14, None),
        (-109.518, 2.86, (1.69680, 55.5), 34.06, None),
        (-53.092, 11.79, AIR, 34.38, None),
        (-29.766, 1.70, (1.59270, 35.3), 33.78, None),
        (-114.300, 11.66, AIR, 36.27, None),
    ]
    return _table(rows)


def _table(rows):
    out = []
    for R, t, glass, diam, asph in rows:
        if R == "stop":
            out.append(_row(SURF_STOP, 0.0, t, glass, diam / 2))
        else:
            out.append(_row(SURF_REFRACT, R, t, glass, diam / 2, 0.0,
                            asph if asph is not None else (0, 0, 0, 0, 0)))
    return np.stack(out)


# --------------------------------------------------------------------------
# PSF request sets.  A request is (field height mm, depth mm, wavelength nm,
# pupil grid N, patch size ks).  Field heights are image heights on the
# sensor along +x.
# --------------------------------------------------------------------------
REQ_DTYPE = np.dtype([("h_mm", "f8"), ("depth_mm", "f8"), ("lambda_nm", "f8"),
                      ("n_grid", "i4"), ("ks", "i4"), ("lens", "i4"), ("v_mm", "f8")])


def bank_grid(field_h_mm, depths_mm, lambdas_nm, n_grid, ks):
    """Requests in bank order [field][depth][wavelength]."""
    reqs = []
    for h in field_h_mm:
        for d in depths_mm:
            for lam in lambdas_nm:
                reqs.append((h, d, lam, n_grid, ks, 0, 0.0))
    return np.array(reqs, dtype=REQ_DTYPE)


def bank_grid_quadrant(field_h_mm, depths_mm, lambdas_nm, n_grid, ks):
    """Requests of a first-quadrant 2-D bank, order [x height][y height]
    [depth][wavelength], both axes sampled at field_h_mm."""
    reqs = []
    for hx in field_h_mm:
        for hy in field_h_mm:
            for d in depths_mm:
                for lam in lambdas_nm:
                    reqs.append((hx, d, lam, n_grid, ks, 0, hy))
    return np.array(reqs, dtype=REQ_DTYPE)


def inverse_uniform_depths(d_near_mm, d_far_mm, n):
    """n depths uniform in inverse depth, ascending in depth."""
    inv = np.linspace(1.0 / d_near_mm, 1.0 / d_far_mm, n)
    return 1.0 / inv


def config_singlet():
    """Small case: the f/2 singlet, 8 field heights x 4 depths, 64x64 pupil
    grid, 31x31 patches on a 64x64 sensor at 4 um pitch, 587.6 nm."""
    field = np.linspace(0.0, 0.12, 8)
    depths = np.array([500.0, 800.0, 1500.0, 3000.0])
    return dict(lens=singlet_f2(), focus_mm=1000.0, pitch_mm=0.004,
                sensor_hw=(64, 64), field_h_mm=field, depths_mm=depths,
                lambdas_nm=np.array([LAMBDA_D]), n_grid=64, ks=31)


def config_full_forward():
    """Full forward: the f/1.8 doublet pair, 32 field heights (0 .. sensor
    half-diagonal) x 32 depths (0.3-3 m uniform in 1/d) x 3 wavelengths,
    256x256 pupil grid, 65x65 patches, 1024x1024 sensor at 2 um pitch."""
    pitch = 0.002
    H = W = 1024
    half_diag = 0.5 * math.hypot(H, W) * pitch
    field = np.linspace(0.0, half_diag, 32)
    depths = inverse_uniform_depths(300.0, 3000.0, 32)
    return dict(lens=doublet_pair_f18(), focus_mm=1000.0, pitch_mm=pitch,
                sensor_hw=(H, W), field_h_mm=field, depths_mm=depths,
                lambdas_nm=np.array(RGB_LAMBDAS_NM), n_grid=256, ks=65)


def config_differentiation():
    """Differentiation: the full-forward lens and bank grid at 128x128 pupil
    samples; render backward over a batch of 8 RGB 512x512 images."""
    c = config_full_forward()
    c.update(n_grid=128, batch=8, image_hw=(512, 512))
    return c


def config_precision():
    """Precision at full resolution: 64 field heights x 64 depths x 3
    wavelengths of 65x65 PSFs (128x128 pupil samples), a batch of 16 RGB
    2048x1536 images at 2 um pitch."""
    pitch = 0.002
    H, W = 2048, 1536
    half_diag = 0.5 * math.hypot(H, W) * pitch
    return dict(lens=doublet_pair_f18(), focus_mm=1000.0, pitch_mm=pitch,
                field_h_mm=np.linspace(0.0, half_diag, 64),
                depths_mm=inverse_uniform_depths(300.0, 3000.0, 64),
                lambdas_nm=np.array(RGB_LAMBDAS_NM), n_grid=128, ks=65, batch=16,
                image_hw=(H, W))


def flip_batch(aif_bases, depth_bases, n):
    """n (image, depth) pairs from a few base maps by flips and channel
    rotations (cheap distinct members of a large batch): image i takes base
    i % len, flip (i // 2) % 4 and channel rotation i // 8; its depth map
    takes another base/flip combination."""
    na, nd = len(aif_bases), len(depth_bases)
    c = aif_bases[0].shape[0]
    aif = np.empty((n,) + aif_bases[0].shape, dtype=aif_bases[0].dtype)
    dep = np.empty((n,) + depth_bases[0].shape, dtype=depth_bases[0].dtype)

    def flip(x, k):
        if k & 1:
            x = x[..., :, ::-1]
        if k & 2:
            x = x[..., ::-1, :]
        return x

    for i in range(n):
        a = flip(aif_bases[i % na], (i // 2) % 4)
        aif[i] = np.roll(a, (i // 8) % c, axis=0)
        dep[i] = flip(depth_bases[(i // 2) % nd], (i + 1) % 4)
    return aif, dep


def pixel_centres_mm(rows, cols, H, W, pitch_mm):
    """Sensor-plane coordinates (x along columns, y along rows) of pixel
    centres relative to the sensor centre (= the optical axis)."""
    x = (np.asarray(cols, dtype=np.float64) - 0.5 * (W - 1)) * pitch_mm
    y = (np.asarray(rows, dtype=np.float64) - 0.5 * (H - 1)) * pitch_mm
    return x, y


def map_requests(depth_m, rows, cols, pitch_mm, lambda_nm, n_grid, ks):
    """Requests of a per-pixel PSF map: one per listed pixel (rows, cols) of
    the (H, W) depth map, at the pixel's 2-D sensor position and depth."""
    H, W = depth_m.shape
    x, y = pixel_centres_mm(rows, cols, H, W, pitch_mm)
    out = np.zeros(len(x), dtype=REQ_DTYPE)
    out["h_mm"], out["v_mm"] = x, y
    out["depth_mm"] = depth_m[np.asarray(rows), np.asarray(cols)].astype(np.float64) * 1000.0
    out["lambda_nm"], out["n_grid"], out["ks"] = lambda_nm, n_grid, ks
    return out


def config_paper_rf50():
    """The paper's own timed workload (Sec. 5.1 implementation details, Table
    S3): Canon RF50mm (Table S1) stopped down to F/4, 550 nm, focus 1 m, a
    24 x 36 mm DP sensor of 512 x 768 pixels, a DP PSF for every pixel of a
    depth map over 0.5-20 m, a 64 x 64 pupil grid (4096 samples) and 21 x 21
    patches."""
    H, W = 512, 768
    return dict(lens=canon_rf50(), f_number=4.0, lambda_nm=550.0, focus_mm=1000.0,
                pitch_mm=36.0 / W, sensor_hw=(H, W), n_grid=64, ks=21,
                d_near_m=0.5, d_far_m=20.0)


def random_requests(n_req, seed=3, n_lenses=2, field_max_mm=1.448,
                    d_near_mm=300.0, d_far_mm=3000.0):
    """Uneven requests: N log-uniform in [32, 512], ks uniform over
    {15, 31, 65, 127}, field/depth/wavelength uniform, lens index uniform."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(math.log(32), math.log(512), size=n_req)).astype(np.int32)
    n = np.clip(n, 32, 512)
    ks = rng.choice(np.array([15, 31, 65, 127], dtype=np.int32), size=n_req)
    h = rng.uniform(0.0, field_max_mm, size=n_req)
    inv = rng.uniform(1.0 / d_far_mm, 1.0 / d_near_mm, size=n_req)
    lam = rng.choice(np.array(RGB_LAMBDAS_NM), size=n_req)
    lens = rng.integers(0, n_lenses, size=n_req).astype(np.int32)
    out = np.zeros(n_req, dtype=REQ_DTYPE)
    out["h_mm"], out["depth_mm"], out["lambda_nm"] = h, 1.0 / inv, lam
    out["n_grid"], out["ks"], out["lens"] = n, ks, lens
    return out


# --------------------------------------------------------------------------
# Scenes
# --------------------------------------------------------------------------
def _gauss_blur_replicate(img, sigma):
    """Separable Gaussian blur truncated at 3 sigma with replicate edges."""
    rad = int(math.ceil(3 * sigma))
    x = np.arange(-rad, rad + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    k /= k.sum()
    p = np.pad(img, ((rad, rad), (0, 0)), mode="edge")
    tmp = sum(k[i] * p[i:i + img.shape[0], :] for i in range(2 * rad + 1))
    p = np.pad(tmp, ((0, 0), (rad, rad)), mode="edge")
    return sum(k[i] * p[:, i:i + img.shape[1]] for i in range(2 * rad + 1))


def aif_blurred_uniform(h, w, seed=0, sigma=1.0):
    """Grayscale (1, 1, h, w) uniform [0, 1] noise blurred by a Gaussian."""
    rng = np.random.default_rng(seed)
    img = rng.uniform(0.0, 1.0, size=(h, w))
    return _gauss_blur_replicate(img, sigma)[None, None]


def aif_pink(n, c, h, w, seed=1):
    """(n, c, h, w) noise with a 1/f amplitude spectrum, each plane rescaled
    to [0, 1]."""
    rng = np.random.default_rng(seed)
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.rfftfreq(w)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    f[0, 0] = 1.0
    out = np.empty((n, c, h, w))
    for i in range(n):
        for j in range(c):
            white = rng.standard_normal((h, w))
            spec = np.fft.rfft2(white) / f
            spec[0, 0] = 0.0
            img = np.fft.irfft2(spec, s=(h, w))
            lo, hi = img.min(), img.max()
            out[i, j] = (img - lo) / (hi - lo)
    return out


def _perlin_octave(h, w, cells, rng):
    """One octave of 2-D gradient noise on a (cells+1)^2 lattice."""
    ang = rng.uniform(0, 2 * math.pi, size=(cells + 1, cells + 1))
    gx, gy = np.cos(ang), np.sin(ang)
    ys = (np.arange(h) + 0.5) / h * cells
    xs = (np.arange(w) + 0.5) / w * cells
    y0 = np.floor(ys).astype(int)
    x0 = np.floor(xs).astype(int)
    fy = (ys - y0)[:, None]
    fx = (xs - x0)[None, :]
    y0 = y0[:, None]
    x0 = x0[None, :]

    def dot(iy, ix, dy, dx):
        return gx[iy, ix] * dx + gy[iy, ix] * dy

    n00 = dot(y0, x0, fy, fx)
    n01 = dot(y0, x0 + 1, fy, fx - 1)
    n10 = dot(y0 + 1, x0, fy - 1, fx)
    n11 = dot(y0 + 1, x0 + 1, fy - 1, fx - 1)
    sy = fy * fy * fy * (fy * (fy * 6 - 15) + 10)
    sx = fx * fx * fx * (fx * (fx * 6 - 15) + 10)
    a = n00 + sx * (n01 - n00)
    b = n10 + sx * (n11 - n10)
    return a + sy * (b - a)


def depth_perlin(n, h, w, seed=2, d_near_m=0.3, d_far_m=3.0, octaves=4,
                 base_cells=4):
    """(n, h, w) smooth random depth in metres: `octaves` octaves of gradient
    noise (base lattice `base_cells` cells across, persistence 0.5), each map
    rescaled linearly to [d_near, d_far]."""
    rng = np.random.default_rng(seed)
    out = np.empty((n, h, w))
    for i in range(n):
        acc = np.zeros((h, w))
        amp = 1.0
        for o in range(octaves):
            acc += amp * _perlin_octave(h, w, base_cells * (2 ** o), rng)
            amp *= 0.5
        lo, hi = acc.min(), acc.max()
        out[i] = d_near_m + (acc - lo) / (hi - lo) * (d_far_m - d_near_m)
    return out


def depth_two_planes(h, w, split_col, near_m, far_m):
    """(1, h, w) depth: near_m for columns < split_col, far_m otherwise."""
    d = np.full((1, h, w), far_m)
    d[:, :, :split_col] = near_m
    return d
