"""FP64 CPU oracle of the Sdirt DP simulator hot path (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's ``cpu_baseline`` /
reference legs may import this package.  It wraps ``sdirt_oracle.cpp`` (plain
FP64 C++, no code shared with the CUDA library) through ctypes.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  lens_info        paraxial EFL/BFL pinned by the thick-lens closed form and
                   by the back focal lengths printed in Tables S1/S2
  trace_hits       pinned by paraxial limits, n sin(theta) across flat
                   interfaces, unit directions, sphere/asphere residuals,
                   reversibility, on-axis symmetry
  psf_bank         pinned by exact integer symmetry (L(a,b) = R(ks-1-a,b) on
                   axis), the degenerate DP sensor (plain histogram), the
                   literal boundary-line test of Eq. (1)/(2), energy bookkeeping
                   and disparity sign; absolute PSF shapes of the aspheric lens
                   are "parity unpinned" beyond these properties
  trace_grad       pinned by FP64 central differences of trace_functional
  mlp_psf          pinned through all five hidden layers by signed, scaled
                   permutation networks whose outputs follow one path back
                   to one input (a transposed weight, a dropped layer, a
                   missing ReLU, a wrong input order, a missing clamp or a
                   per-plane normalisation each fail a pin), by a bias chain
                   through every layer, the biases-only closed form and the
                   normalised-input corners
  render_*         pinned by the delta-PSF and constant-image identities, a
                   shift-invariant kernel against scipy correlation and brute
                   force of the supplement's unfold/fold formulation; the
                   quadrant bank against a per-pixel map of PSFs traced at
                   each pixel's own signed field point
  render_bank_bwd  pinned by the adjoint identities <G, R(I, B)> =
                   <R*_I(G), I> = <R*_B(G), B> against the forward (radial
                   and quadrant banks) and by central differences of it
  render_select    pinned by a brute-force nearest-height / depth-bracket
                   search
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "sdirt_oracle.cpp"
_LIB_PATH = _HERE / "_build" / "libsdirt_oracle.so"

# stats slots per request
STATS = ("launched", "reached", "L", "R", "dp_missed", "clipped", "vignetted", "other")
# ray states
R_OK, R_MISS, R_CLIP, R_TIR, R_NEWTON, R_BACK = range(6)
# bank field layouts: radial heights, or a first-quadrant grid used through
# the PSF's flip symmetry about both axes
FIELD_RADIAL, FIELD_QUADRANT = 0, 1
# PSF accumulation modes and normalisations
MODE_HARD, MODE_BILINEAR = 0, 1
NORM_NONE, NORM_JOINT, NORM_SEPARATE, NORM_PER_RAY = 0, 1, 2, 3
NPAR_SURF = 8


def build(force: bool = False) -> Path:
    """Compile the oracle with g++ (-O2, no FP contraction)."""
    if (not force and _LIB_PATH.exists()
            and _LIB_PATH.stat().st_mtime >= _SRC.stat().st_mtime):
        return _LIB_PATH
    _LIB_PATH.parent.mkdir(parents=True, exist_ok=True)
    tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp")
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", str(tmp), str(_SRC), "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(str(build()))
        P = ctypes.POINTER
        d, i, f = ctypes.c_double, ctypes.c_int, ctypes.c_float
        pd, pi, pf = P(d), P(i), P(f)
        pl = P(ctypes.c_int64)
        L.or_lens_info.argtypes = [pd, i, d, d, d, pd]
        L.or_trace_hits.argtypes = [pd, i, d, pd, pd, pd, i, pi]
        L.or_psf_bank.argtypes = [pd, i, d, pd, i, pd, i, i, pd, pl, i]
        L.or_trace_functional.argtypes = [pd, i, d, pd, i, pd, pd, pi, pd, i, i, pd]
        L.or_trace_grad.argtypes = [pd, i, d, pd, i, pd, pd, pi, i, pd, i]
        L.or_render_bank.argtypes = [pd, i, i, i, i, pf, pd, i, i, i, i, pf, pf, f, pd, i]
        L.or_render_map.argtypes = [pd, i, i, i, i, pd, i, pd]
        L.or_render_bank_bwd.argtypes = [pd, pd, i, i, i, i, pf, pd, i, i, i, i,
                                         pf, pf, f, pd, pd]
        L.or_render_select.argtypes = [i, i, pf, pf, i, pf, i, f, pd]
        L.or_render_bank_pixels.argtypes = [pd, i, i, i, i, pf, pd, i, i, i, i, pf, pf, f,
                                            pi, i, pd, i]
        L.or_render_bank_bwd_mode.argtypes = [pd, pd, i, i, i, i, pf, pd, i, i, i, i,
                                              pf, pf, f, i, pd, pd]
        L.or_render_bank_mode.argtypes = [pd, i, i, i, i, pf, pd, i, i, i, i, pf, pf, f, i,
                                          pd, i]
        L.or_render_bank_pixels_mode.argtypes = [pd, i, i, i, i, pf, pd, i, i, i, i, pf, pf,
                                                 f, i, pi, i, pd, i]
        for fn in ("or_lens_info", "or_trace_hits", "or_psf_bank", "or_trace_functional",
                   "or_trace_grad", "or_render_bank", "or_render_map",
                   "or_render_bank_bwd", "or_render_select", "or_render_bank_pixels",
                   "or_render_bank_mode", "or_render_bank_pixels_mode",
                   "or_render_bank_bwd_mode"):
            getattr(L, fn).restype = i
        _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pf(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _pi(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def lens_info(table, focus_mm=1000.0, lambda_nm=587.5618, depth_mm=1000.0):
    """Paraxial data: dict(efl, bfl, z_ep, r_ep, sensor_dist, m_sensor,
    img_dist, z_sensor)."""
    t = _f64(table)
    out = np.zeros(8)
    _check(lib().or_lens_info(_pd(t), t.shape[0], focus_mm, lambda_nm, depth_mm,
                              _pd(out)), "lens_info")
    keys = ("efl", "bfl", "z_ep", "r_ep", "sensor_dist", "m_sensor", "img_dist", "z_sensor")
    return dict(zip(keys, out.tolist()))


def _req_rows(reqs):
    """Structured request array (workloads.REQ_DTYPE) -> (n, 6) float64 rows
    (h_mm, depth_mm, lambda_nm, n_grid, ks, v_mm); v_mm is 0 when absent."""
    r = np.zeros((len(reqs), 6))
    r[:, 0] = reqs["h_mm"]
    r[:, 1] = reqs["depth_mm"]
    r[:, 2] = reqs["lambda_nm"]
    r[:, 3] = reqs["n_grid"]
    r[:, 4] = reqs["ks"]
    if "v_mm" in reqs.dtype.names:
        r[:, 5] = reqs["v_mm"]
    return r


def _sensor(sensor):
    return _f64([sensor["ps"], sensor["h"], sensor["f"], sensor["w"], sensor["r"]])


HIT_FIELDS = ("x", "y", "dx", "dy", "dz", "state", "side", "clipped", "a", "b",
              "margin", "surf")


def trace_hits(table, focus_mm, req, sensor):
    """Per-ray records of one request (single structured element)."""
    t = _f64(table)
    r = _req_rows(np.atleast_1d(req))[0].copy()
    n = int(r[3])
    out = np.zeros((n * n, 12))
    k = ctypes.c_int(0)
    _check(lib().or_trace_hits(_pd(t), t.shape[0], focus_mm, _pd(r), _pd(_sensor(sensor)),
                               _pd(out), n * n, ctypes.byref(k)), "trace_hits")
    out = out[:k.value]
    return {name: out[:, j] for j, name in enumerate(HIT_FIELDS)}


def psf_bank(table, focus_mm, reqs, sensor, mode=MODE_HARD, norm=NORM_JOINT,
             n_threads=1):
    """PSFs of all requests: list of (2, ks, ks) arrays and (n_req, 8) stats."""
    t = _f64(table)
    r = _req_rows(reqs)
    ks = r[:, 4].astype(int)
    total = int((2 * ks * ks).sum())
    bank = np.zeros(total)
    stats = np.zeros((len(reqs), len(STATS)), dtype=np.int64)
    _check(lib().or_psf_bank(_pd(t), t.shape[0], focus_mm, _pd(r), len(reqs),
                             _pd(_sensor(sensor)), mode, norm, _pd(bank),
                             stats.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             n_threads), "psf_bank")
    out, off = [], 0
    for k in ks:
        out.append(bank[off:off + 2 * k * k].reshape(2, k, k))
        off += 2 * k * k
    return out, stats


def trace_functional(table, focus_mm, reqs, sensor, G, pids=(), delta=(), freeze=True):
    """sum_i <G_i, PSF_i> for per-ray-normalised bilinear PSFs of the lens
    perturbed by delta on parameters pids (ray generation at nominal)."""
    t = _f64(table)
    r = _req_rows(reqs)
    g = _f64(np.concatenate([np.ravel(x) for x in G]))
    p = np.ascontiguousarray(pids, dtype=np.int32)
    dl = _f64(delta) if len(delta) else np.zeros(1)
    out = np.zeros(1)
    _check(lib().or_trace_functional(_pd(t), t.shape[0], focus_mm, _pd(r), len(reqs),
                                     _pd(_sensor(sensor)), _pd(g), _pi(p), _pd(dl),
                                     len(p), int(freeze), _pd(out)), "trace_functional")
    return float(out[0])


def trace_grad(table, focus_mm, reqs, sensor, G, pids, n_threads=1):
    """d/dtheta of trace_functional at delta = 0 (dual numbers)."""
    t = _f64(table)
    r = _req_rows(reqs)
    g = _f64(np.concatenate([np.ravel(x) for x in G]))
    p = np.ascontiguousarray(pids, dtype=np.int32)
    out = np.zeros(len(p))
    _check(lib().or_trace_grad(_pd(t), t.shape[0], focus_mm, _pd(r), len(reqs),
                               _pd(_sensor(sensor)), _pd(g), _pi(p), len(p), _pd(out),
                               n_threads), "trace_grad")
    return out


def param_id(surface, which):
    """Parameter id: which in ('c', 'k', 'a4', 'a6', 'a8', 'a10', 'a12', 't')."""
    j = {"c": 0, "k": 1, "a4": 2, "a6": 3, "a8": 4, "a10": 5, "a12": 6, "t": 7}[which]
    return surface * NPAR_SURF + j


def _bank_fields(b, field_h_mm, field_mode):
    """Heights per axis of a bank: radial (F,Z,...) or quadrant (F*F,Z,...)."""
    cells = b.shape[0]
    F = len(field_h_mm)
    if cells != (F * F if field_mode == FIELD_QUADRANT else F):
        raise ValueError("bank field cells do not match field_h_mm and field_mode")
    return F


def render_bank(aif, depth_m, bank, field_h_mm, depths_m, pitch_mm, n_threads=1,
                field_mode=0):
    """aif (N,C,H,W); depth (N,H,W) m; bank (F,Z,NL,2,ks,ks) -> (N,2C,H,W).
    field_mode=FIELD_QUADRANT: bank (F*F,Z,NL,2,ks,ks) over the first
    quadrant (cell ix*F + iy), used through the PSF's flip symmetry."""
    a = _f64(aif)
    N, C, H, W = a.shape
    dm = _f32(depth_m)
    b = _f64(bank)
    _, Z, NL, _, ks, _ = b.shape
    F = _bank_fields(b, field_h_mm, field_mode)
    out = np.zeros((N, 2 * C, H, W))
    _check(lib().or_render_bank_mode(_pd(a), N, C, H, W, _pf(dm), _pd(b), F, Z, NL, ks,
                                     _pf(_f32(field_h_mm)), _pf(_f32(depths_m)),
                                     float(np.float32(pitch_mm)), field_mode, _pd(out),
                                     n_threads), "render_bank")
    return out


def render_bank_pixels(aif, depth_m, bank, field_h_mm, depths_m, pitch_mm, pix, n_threads=1,
                       field_mode=0):
    """Bank-mode render of the pixels pix (k, 3) = (n, y, x) -> (k, 2C)."""
    a = _f64(aif)
    N, C, H, W = a.shape
    dm = _f32(depth_m)
    b = _f64(bank)
    _, Z, NL, _, ks, _ = b.shape
    F = _bank_fields(b, field_h_mm, field_mode)
    px = np.ascontiguousarray(pix, dtype=np.int32)
    out = np.zeros((len(px), 2 * C))
    _check(lib().or_render_bank_pixels_mode(_pd(a), N, C, H, W, _pf(dm), _pd(b), F, Z, NL, ks,
                                            _pf(_f32(field_h_mm)), _pf(_f32(depths_m)),
                                            float(np.float32(pitch_mm)), field_mode, _pi(px),
                                            len(px), _pd(out), n_threads), "render_bank_pixels")
    return out


def render_map(aif, psf_map):
    """aif (N,C,H,W); psf_map (H,W,2,ks,ks) -> (N,2C,H,W)."""
    a = _f64(aif)
    N, C, H, W = a.shape
    m = _f64(psf_map)
    ks = m.shape[-1]
    out = np.zeros((N, 2 * C, H, W))
    _check(lib().or_render_map(_pd(a), N, C, H, W, _pd(m), ks, _pd(out)), "render_map")
    return out


def render_bank_bwd(grad_out, aif, depth_m, bank, field_h_mm, depths_m, pitch_mm,
                    field_mode=0):
    """Adjoint of render_bank: (grad_aif, grad_bank)."""
    g = _f64(grad_out)
    a = _f64(aif)
    N, C, H, W = a.shape
    dm = _f32(depth_m)
    b = _f64(bank)
    _, Z, NL, _, ks, _ = b.shape
    F = _bank_fields(b, field_h_mm, field_mode)
    ga = np.zeros_like(a)
    gb = np.zeros_like(b)
    _check(lib().or_render_bank_bwd_mode(_pd(g), _pd(a), N, C, H, W, _pf(dm), _pd(b), F, Z,
                                         NL, ks, _pf(_f32(field_h_mm)), _pf(_f32(depths_m)),
                                         float(np.float32(pitch_mm)), field_mode, _pd(ga),
                                         _pd(gb)), "render_bank_bwd")
    return ga, gb


def render_select(depth_m, field_h_mm, depths_m, pitch_mm):
    """Per-pixel (f, z0, z1, t) of a single (H, W) depth map."""
    dm = _f32(depth_m)
    H, W = dm.shape
    out = np.zeros((H, W, 4))
    fh = _f32(field_h_mm)
    dz = _f32(depths_m)
    _check(lib().or_render_select(H, W, _pf(dm), _pf(fh), len(fh), _pf(dz), len(dz),
                                  float(np.float32(pitch_mm)), _pd(out)), "render_select")
    return out


# --------------------------------------------------------------------------
# DP PSF prediction network (Sec. 3.2, "Pixel-wise DP image rendering
# module"; Sec. 5.1 implementation details)
# --------------------------------------------------------------------------
def mlp_inputs(depth_m, d_min_m, d_max_m):
    """Normalised object point p = (x_n, y_n, d_n) of every pixel of a depth
    map (H, W), row-major -> (H*W, 3): the pixel's sensor position scaled to
    [-1, 1] (the frustum's x and y at its depth, Sec. 3.2) and the depth
    scaled linearly from [d_min, d_max] to [-1, 1]."""
    d = np.asarray(depth_m, dtype=np.float64)
    H, W = d.shape
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    xn = (x - 0.5 * (W - 1)) / (0.5 * W)
    yn = (y - 0.5 * (H - 1)) / (0.5 * H)
    dn = 2.0 * (d - d_min_m) / (d_max_m - d_min_m) - 1.0
    return np.stack([xn, yn, dn], -1).reshape(-1, 3)


def mlp_psf(weights, biases, p, ks):
    """The network of Sec. 3.2 in FP64: h = ReLU(W_l h + b_l) for the input
    layer and the hidden layers (l = 0..4, 512 neurons each), o = W_5 h + b_5
    with 2 ks^2 outputs; at inference o is clamped at 0 and divided by its
    sum (the sum normalisation of Sec. 3.2, joint over L and R).
    p (n, 3) -> (n, 2, ks, ks)."""
    h = np.asarray(p, dtype=np.float64)
    for l in range(5):
        h = np.maximum(h @ np.asarray(weights[l], np.float64).T + np.asarray(biases[l], np.float64),
                       0.0)
    o = h @ np.asarray(weights[5], np.float64).T + np.asarray(biases[5], np.float64)
    o = np.maximum(o, 0.0)
    s = o.sum(axis=1, keepdims=True)
    o = np.divide(o, s, out=np.zeros_like(o), where=s > 0)
    return o.reshape(-1, 2, ks, ks)
