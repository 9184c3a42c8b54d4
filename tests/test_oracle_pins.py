"""Pins of the FP64 oracle against what optics and the paper fix (no GPU).

Each test checks the oracle against something other than itself: closed
forms, values printed in the paper (tests/golden), exact symmetries, brute
force over the oracle's own per-ray records, and library routines.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from golden.load import paper_values

LAM_D = W.LAMBDA_D


def dp_sensor(ps, h=W.DP_H, f=W.DP_F, w=W.DP_W, r=W.DP_R):
    return dict(ps=ps, h=h * ps, f=f * ps, w=w * ps, r=r * ps)


def one_req(h, d, lam=LAM_D, n=64, ks=31):
    return W.bank_grid([h], [d], [lam], n, ks)[0]


# --------------------------------------------------------------------------
# P1 paraxial
# --------------------------------------------------------------------------
def test_singlet_thick_lens_closed_form():
    """Sec. 3.1 lens model: EFL/BFL/image distance of the f/2 singlet equal
    the thick-lens formulas (principal planes, Gaussian imaging)."""
    n, R1, R2, t = 1.5168, 51.68, -51.68, 5.0
    phi = (n - 1) * (1 / R1 - 1 / R2 + (n - 1) * t / (n * R1 * R2))
    f = 1 / phi
    bfl = f * (1 - (n - 1) * t / (n * R1))
    dH = -f * (n - 1) * t / (n * R2)      # front principal plane from V1
    dHp = -f * (n - 1) * t / (n * R1)     # back principal plane from V2
    so = 1000.0 + dH
    si = 1 / (1 / f - 1 / so)
    info = O.lens_info(W.singlet_f2(), 1000.0, LAM_D, 1000.0)
    assert info["efl"] == pytest.approx(f, rel=1e-12)
    assert info["bfl"] == pytest.approx(bfl, rel=1e-12)
    assert info["sensor_dist"] == pytest.approx(si + dHp, rel=1e-12)
    assert info["efl"] == pytest.approx(50.838, abs=1e-3)
    # stop in the first vertex plane: the entrance pupil is the stop itself
    assert info["z_ep"] == 0.0 and info["r_ep"] == 12.5


def test_paper_lenses_bfl_and_f_number():
    """Tables S1/S2: the printed last thickness is the paraxial back focal
    distance, and EFL / entrance-pupil diameter is the lenses' F/1.8."""
    g = paper_values()
    for tab, key_t, key_f in ((W.canon_rf50(), "rf50_last_thickness_mm", "rf50_f_number"),
                              (W.canon_rf35(), "rf35_last_thickness_mm", "rf35_f_number")):
        info = O.lens_info(tab, 0.0, LAM_D, 1e12)
        assert info["bfl"] == pytest.approx(g[key_t], abs=0.015)
        fno = info["efl"] / (2 * info["r_ep"])
        assert fno == pytest.approx(g[key_f], rel=0.04)


def test_cauchy_fit_matches_abbe_definition():
    """Reading of the glass columns: n(d) = nd and (nF - nC) = (nd-1)/Vd.
    Checked through the paraxial power of a thin plano-convex element."""
    R = 100.0
    tab = np.stack([W._row(W.SURF_STOP, 0, 0, W.AIR, 5.0),
                    W._row(W.SURF_REFRACT, R, 1e-9, W.CROWN, 10.0),
                    W._row(W.SURF_REFRACT, 0.0, 100.0, W.AIR, 10.0)])
    nd, vd = W.CROWN
    n = {}
    for lam in (W.LAMBDA_F, W.LAMBDA_D, W.LAMBDA_C):
        efl = O.lens_info(tab, 0.0, lam, 1e12)["efl"]
        n[lam] = 1 + R / efl  # thin plano-convex: 1/f = (n-1)/R
    assert n[W.LAMBDA_D] == pytest.approx(nd, abs=1e-9)
    assert n[W.LAMBDA_F] - n[W.LAMBDA_C] == pytest.approx((nd - 1) / vd, rel=1e-7)


# --------------------------------------------------------------------------
# P2/P3 real-ray trace
# --------------------------------------------------------------------------
def single_surface(c, k=0.0, asph=(0, 0, 0, 0, 0), n_glass=1.6, z_sensor=30.0):
    R = 0.0 if c == 0 else 1.0 / c
    return np.stack([W._row(W.SURF_STOP, 0, 0, W.AIR, 4.0),
                     W._row(W.SURF_REFRACT, R, z_sensor, (n_glass, 0.0), 50.0, k, asph)])


def sag_and_slope(rho, c, k, a):
    """Even-asphere sag and its radial slope, written out term by term."""
    q = np.sqrt(1 - (1 + k) * c * c * rho * rho)
    z = c * rho ** 2 / (1 + q) + sum(a[j] * rho ** (2 * j + 4) for j in range(5))
    dz = c * rho / q + sum((2 * j + 4) * a[j] * rho ** (2 * j + 3) for j in range(5))
    return z, dz


@pytest.mark.parametrize("c,k,a", [
    (1 / 40.0, 0.0, (0, 0, 0, 0, 0)),                       # sphere, closed form
    (1 / 40.0, -0.6, (0, 0, 0, 0, 0)),                      # conic, closed form
    (1 / 40.0, -0.6, (2e-4, -3e-6, 1e-8, -2e-10, 1e-12)),   # full even asphere
    (0.0, 0.0, (1e-3, 0, 0, 0, 0)),                         # pure a4 "plate"
    (-1 / 60.0, 0.3, (-1e-4, 2e-6, 0, 0, 0)),               # concave asphere
])
def test_single_surface_collimated_closed_form(c, k, a):
    """A collimated beam on one surface: hit at z = sag(rho), incidence
    angle atan(dsag/drho), Snell sin(ti) = n sin(tt), straight line to the
    sensor -- the textbook meridional trace, for every ray of the grid."""
    n2, zs = 1.6, 30.0
    tab = single_surface(c, k, a, n2, zs)
    req = one_req(0.0, 1e13, n=16, ks=3)
    hits = O.trace_hits(tab, 0.0, req, dp_sensor(0.004))
    assert np.all(hits["state"] == O.R_OK)
    N = 16
    ix, iy = np.meshgrid(np.arange(N), np.arange(N))
    keep = (2 * ix + 1 - N) ** 2 + (2 * iy + 1 - N) ** 2 <= N * N
    ex = ((2 * ix + 1 - N) / N * 4.0)[keep]
    ey = ((2 * iy + 1 - N) / N * 4.0)[keep]
    rho = np.hypot(ex, ey)
    z, slope = sag_and_slope(rho, c, k, a)
    ti = np.arctan(slope)
    tt = np.arcsin(np.sin(ti) / n2)
    rho_s = rho - (zs - z) * np.tan(ti - tt)
    np.testing.assert_allclose(hits["x"], rho_s * ex / rho, atol=1e-9)
    np.testing.assert_allclose(hits["y"], rho_s * ey / rho, atol=1e-9)
    d = np.sqrt(hits["dx"] ** 2 + hits["dy"] ** 2 + hits["dz"] ** 2)
    np.testing.assert_allclose(d, 1.0, atol=1e-13)


def test_newton_path_equals_closed_form_sphere():
    """A negligible a12 forces the Newton path; it must land where the closed
    form conic intersection lands."""
    base = W.doublet_pair_f18()
    base[:, W.COL_A4:] = 0.0
    base[:, W.COL_K] = 0.0
    newton = base.copy()
    newton[1:, W.COL_A4 + 4] = 1e-40
    req = one_req(0.8, 700.0, n=32, ks=65)
    S = dp_sensor(0.002)
    h0 = O.trace_hits(base, 1000.0, req, S)
    h1 = O.trace_hits(newton, 1000.0, req, S)
    np.testing.assert_allclose(h1["x"], h0["x"], atol=1e-12)
    np.testing.assert_allclose(h1["y"], h0["y"], atol=1e-12)


def test_plane_parallel_plate():
    """Flat interfaces: n sin(theta) is conserved, so a plate leaves the
    direction unchanged and, on a plane normal to the axis, shifts the ray by
    t (tan(th) - tan(th')) with sin(th') = sin(th) / n relative to the
    straight line."""
    n, t, zs = 1.7, 10.0, 25.0
    tab = np.stack([W._row(W.SURF_STOP, 0, 0, W.AIR, 3.0),
                    W._row(W.SURF_REFRACT, 0.0, t, (n, 0.0), 30.0),
                    W._row(W.SURF_REFRACT, 0.0, zs - t, W.AIR, 30.0)])
    air = tab.copy()
    air[1, W.COL_ND] = 1.0
    # same object point for both: x_o = h / m_sensor of each lens
    m_p = O.lens_info(tab, 0.0, LAM_D, 200.0)["m_sensor"]
    m_a = O.lens_info(air, 0.0, LAM_D, 200.0)["m_sensor"]
    xo = 0.5 / m_a
    S = dp_sensor(0.004)
    hp = O.trace_hits(tab, 0.0, one_req(xo * m_p, 200.0, n=8, ks=3), S)
    ha = O.trace_hits(air, 0.0, one_req(0.5, 200.0, n=8, ks=3), S)
    for comp in ("dx", "dy", "dz"):
        np.testing.assert_allclose(hp[comp], ha[comp], atol=1e-15)
    sin_t = np.sqrt(ha["dx"] ** 2 + ha["dy"] ** 2)
    cos_t = ha["dz"]
    shift = t * (sin_t / cos_t - sin_t / np.sqrt(n * n - sin_t ** 2))
    ux, uy = ha["dx"] / sin_t, ha["dy"] / sin_t
    np.testing.assert_allclose(ha["x"] - hp["x"], shift * ux, atol=1e-12)
    np.testing.assert_allclose(ha["y"] - hp["y"], shift * uy, atol=1e-12)


def test_small_pupil_lands_on_paraxial_image_point():
    """As the pupil shrinks, the real rays' centroid converges to the
    paraxial chief-ray landing point (h, 0) on the sensor.  What remains is
    distortion, third order in the field: e(2h) = 8 e(h) to leading order.
    At the focus depth the whole spot collapses."""
    for tab in (W.singlet_f2(), W.doublet_pair_f18()):
        tiny = tab.copy()
        tiny[0, W.COL_SD] = 1e-4
        for d in (500.0, 1000.0, 3000.0):
            err = {}
            for h in (0.0, 0.03, 0.06):
                hits = O.trace_hits(tiny, 1000.0, one_req(h, d, n=8, ks=3), dp_sensor(0.004))
                assert np.all(hits["state"] == O.R_OK)
                err[h] = hits["x"].mean() - h
                assert abs(hits["y"].mean()) < 1e-15
                if d == 1000.0:
                    assert np.abs(hits["x"] - h).max() < 1e-7
            assert abs(err[0.0]) < 1e-15
            assert abs(err[0.06]) < 1e-5 * 0.06
            assert err[0.06] / err[0.03] == pytest.approx(8.0, rel=0.02)


def test_on_axis_rotational_symmetry():
    """On axis the landing radius depends only on the pupil radius."""
    tab = W.doublet_pair_f18()
    N = 32
    hits = O.trace_hits(tab, 1000.0, one_req(0.0, 600.0, n=N, ks=65), dp_sensor(0.002))
    ix, iy = np.meshgrid(np.arange(N), np.arange(N))
    keep = (2 * ix + 1 - N) ** 2 + (2 * iy + 1 - N) ** 2 <= N * N
    a, b = (2 * ix + 1 - N)[keep], (2 * iy + 1 - N)[keep]
    r = np.hypot(hits["x"], hits["y"])
    lookup = {(ai, bi): ri for ai, bi, ri in zip(a, b, r)}
    for (ai, bi), ri in lookup.items():
        assert abs(lookup[(bi, ai)] - ri) < 1e-12
        assert abs(lookup[(-ai, bi)] - ri) < 1e-12


# --------------------------------------------------------------------------
# P4-P7 binning
# --------------------------------------------------------------------------
def test_on_axis_lr_mirror_exact():
    """On axis, L(a, b) = R(ks-1-a, b) exactly (integer counts) and both are
    symmetric in y (the DP split is along x only)."""
    cfg = W.config_singlet()
    S = dp_sensor(cfg["pitch_mm"])
    reqs = W.bank_grid([0.0], cfg["depths_mm"], cfg["lambdas_nm"], 64, 31)
    psfs, st = O.psf_bank(cfg["lens"], 1000.0, reqs, S, O.MODE_HARD, O.NORM_NONE)
    for p in psfs:
        assert p.sum() > 0
        np.testing.assert_array_equal(p[0], p[1][:, ::-1])
        np.testing.assert_array_equal(p[0], p[0][::-1, :])


def test_energy_bookkeeping():
    """Every launched ray is reached or lost; every reached ray is exactly one
    of L, R, DP-missed, clipped; hard-mode PSF mass equals L + R."""
    cfg = W.config_singlet()
    S = dp_sensor(cfg["pitch_mm"])
    reqs = W.bank_grid(cfg["field_h_mm"][::3], cfg["depths_mm"], cfg["lambdas_nm"], 64, 31)
    psfs, st = O.psf_bank(cfg["lens"], 1000.0, reqs, S, O.MODE_HARD, O.NORM_NONE)
    launched, reached, L, R, miss, clip, vign, other = st.T
    N = 64
    ix, iy = np.meshgrid(np.arange(N), np.arange(N))
    n_in = int(((2 * ix + 1 - N) ** 2 + (2 * iy + 1 - N) ** 2 <= N * N).sum())
    assert np.all(launched == n_in)
    np.testing.assert_array_equal(launched, reached + vign + other)
    np.testing.assert_array_equal(reached, L + R + miss + clip)
    for p, l, r in zip(psfs, L, R):
        assert p[0].sum() == l and p[1].sum() == r


def test_degenerate_sensor_is_plain_histogram():
    """h = 0, w = ps/2, r >= ps/sqrt(2): every ray is inside its microlens and
    s = dx, so L + R is the plain 2-D histogram of the landing points and L the
    histogram of landings in the +x half of their pixel (brute force)."""
    cfg = W.config_full_forward()
    ps = cfg["pitch_mm"]
    S = dict(ps=ps, h=0.0, f=1.44 * ps, w=0.5 * ps, r=0.75 * ps)
    for h, d in ((0.0, 900.0), (0.7, 1200.0), (1.3, 2000.0)):
        req = one_req(h, d, lam=W.LAMBDA_F, n=64, ks=65)
        psfs, _ = O.psf_bank(cfg["lens"], 1000.0, np.array([req]), S, O.MODE_HARD, O.NORM_NONE)
        hits = O.trace_hits(cfg["lens"], 1000.0, req, S)
        ok = hits["state"] == O.R_OK
        fx = (hits["x"][ok] - h) / ps + 32
        fy = hits["y"][ok] / ps + 32
        a, b = np.floor(fx + 0.5).astype(int), np.floor(fy + 0.5).astype(int)
        inside = (a >= 0) & (a < 65) & (b >= 0) & (b < 65)
        plus = (fx - a) >= 0
        hist = np.zeros((2, 65, 65))
        np.add.at(hist[0], (b[inside & plus], a[inside & plus]), 1)
        np.add.at(hist[1], (b[inside & ~plus], a[inside & ~plus]), 1)
        np.testing.assert_array_equal(psfs[0], hist)


def test_side_equals_literal_boundary_lines():
    """Eq. (1)/(2) written literally (boundary lines x_L, x_M, x_R around the
    pixel centre) give the same L/R/miss decision as the oracle."""
    cfg = W.config_full_forward()
    ps = cfg["pitch_mm"]
    S = dp_sensor(ps)
    h_, f_, w_, r_ = S["h"], S["f"], S["w"], S["r"]
    for h, d, lam in ((0.0, 500.0, W.LAMBDA_D), (1.0, 1500.0, W.LAMBDA_C),
                      (0.4, 1000.0, W.LAMBDA_F)):
        req = one_req(h, d, lam=lam, n=96, ks=65)
        hits = O.trace_hits(cfg["lens"], 1000.0, req, S)
        ok = (hits["state"] == O.R_OK) & (hits["margin"] > 1e-12)
        x, y = hits["x"][ok], hits["y"][ok]
        tan = hits["dx"][ok] / hits["dz"][ok]
        a, b = hits["a"][ok], hits["b"][ok]
        xi = h + (a - 32) * ps
        yi = (b - 32) * ps
        inside = (x - xi) ** 2 + (y - yi) ** 2 <= r_ ** 2
        k = h_ / (f_ - h_)
        xL = np.where(inside, xi + w_ - (f_ * tan - w_) * k, xi + w_ - h_ * tan)
        xM = np.where(inside, xi - f_ * tan * k, xi - h_ * tan)
        xR = np.where(inside, xi - w_ - (f_ * tan + w_) * k, xi - w_ - h_ * tan)
        side = np.full(len(x), 2)
        side[(x >= xM) & (x < xL)] = 0
        side[(x >= xR) & (x < xM)] = 1
        np.testing.assert_array_equal(side, hits["side"][ok])
        assert len(x) > 5000


def test_disparity_sign_reverses_across_focus():
    """Sec. 5.3: the L/R phase difference reverses between 0.5 m and 1.5 m
    when focused at 1 m (centroid of L minus centroid of R)."""
    cfg = W.config_full_forward()
    S = dp_sensor(cfg["pitch_mm"])
    reqs = W.bank_grid([0.0, 0.5], [500.0, 1500.0], [W.LAMBDA_D], 128, 65)
    psfs, _ = O.psf_bank(cfg["lens"], 1000.0, reqs, S, O.MODE_HARD, O.NORM_NONE)
    xs = np.arange(65)

    def disp(p):
        cl = (p[0].sum(0) * xs).sum() / p[0].sum()
        cr = (p[1].sum(0) * xs).sum() / p[1].sum()
        return cl - cr

    d = [disp(p) for p in psfs]  # order: (h0, 0.5m), (h0, 1.5m), (h.5, 0.5m), (h.5, 1.5m)
    assert d[0] * d[1] < 0 and d[2] * d[3] < 0
    assert abs(d[0]) > 0.5 and abs(d[1]) > 0.1


def test_normalisations():
    """Joint sum normalisation gives sum(L+R) = 1 and keeps L/R ratio;
    separate gives each 1; per-ray divides by the launched count."""
    cfg = W.config_singlet()
    S = dp_sensor(cfg["pitch_mm"])
    reqs = W.bank_grid([0.06], [800.0], cfg["lambdas_nm"], 64, 31)
    raw, st = O.psf_bank(cfg["lens"], 1000.0, reqs, S, O.MODE_HARD, O.NORM_NONE)
    joint, _ = O.psf_bank(cfg["lens"], 1000.0, reqs, S, O.MODE_HARD, O.NORM_JOINT)
    sep, _ = O.psf_bank(cfg["lens"], 1000.0, reqs, S, O.MODE_HARD, O.NORM_SEPARATE)
    per, _ = O.psf_bank(cfg["lens"], 1000.0, reqs, S, O.MODE_HARD, O.NORM_PER_RAY)
    r = raw[0]
    np.testing.assert_allclose(joint[0], r / r.sum(), rtol=1e-15)
    np.testing.assert_allclose(sep[0][0], r[0] / r[0].sum(), rtol=1e-15)
    np.testing.assert_allclose(sep[0][1], r[1] / r[1].sum(), rtol=1e-15)
    np.testing.assert_allclose(per[0], r / st[0, 0], rtol=1e-15)


def test_bilinear_mode_mass_and_centroid():
    """Bilinear splatting conserves each ray's unit energy when all four taps
    are inside, and places the centroid at the landing point (brute force)."""
    cfg = W.config_full_forward()
    ps = cfg["pitch_mm"]
    S = dp_sensor(ps)
    req = one_req(0.3, 1050.0, n=48, ks=65)
    psf, st = O.psf_bank(cfg["lens"], 1000.0, np.array([req]), S, O.MODE_BILINEAR, O.NORM_NONE)
    hits = O.trace_hits(cfg["lens"], 1000.0, req, S)
    ok = (hits["state"] == O.R_OK) & (hits["side"] < 2)
    fx = (hits["x"][ok] - 0.3) / ps + 32
    fy = hits["y"][ok] / ps + 32
    assert fx.min() > 0 and fx.max() < 64 and fy.min() > 0 and fy.max() < 64
    p = psf[0]
    assert p.sum() == pytest.approx(ok.sum(), rel=1e-12)
    xs = np.arange(65)
    cx = ((p[0] + p[1]).sum(0) * xs).sum() / p.sum()
    assert cx == pytest.approx(fx.mean(), rel=1e-12)
    left = hits["side"][ok] == 0
    assert p[0].sum() == pytest.approx(left.sum(), rel=1e-12)


# --------------------------------------------------------------------------
# P9 gradients of the trace
# --------------------------------------------------------------------------
def test_trace_grad_matches_central_differences():
    """Dual-number gradient of <G, PSF> equals FP64 central differences with
    the discrete decisions frozen (relative step 1e-6)."""
    tab = W.doublet_pair_f18()
    S = dp_sensor(0.002)
    reqs = W.bank_grid([0.0, 0.9], [450.0, 2000.0], [W.LAMBDA_D], 24, 65)
    rng = np.random.default_rng(5)
    G = [rng.standard_normal((2, 65, 65)) for _ in reqs]
    pids = [O.param_id(1, "c"), O.param_id(6, "c"), O.param_id(1, "k"), O.param_id(6, "k"),
            O.param_id(1, "a4"), O.param_id(6, "a6"), O.param_id(2, "t"), O.param_id(6, "t"),
            O.param_id(3, "c")]
    grad = O.trace_grad(tab, 1000.0, reqs, S, G, pids)
    info = O.lens_info(tab, 1000.0)
    nominal = {O.param_id(1, "c"): 1 / tab[1, 1], O.param_id(6, "c"): 1 / tab[6, 1],
               O.param_id(1, "k"): tab[1, 6], O.param_id(6, "k"): tab[6, 6],
               O.param_id(1, "a4"): tab[1, 7], O.param_id(6, "a6"): tab[6, 8],
               O.param_id(2, "t"): tab[2, 2], O.param_id(6, "t"): info["sensor_dist"],
               O.param_id(3, "c"): 1 / tab[3, 1]}
    for j, pid in enumerate(pids):
        hstep = 1e-6 * max(abs(nominal[pid]), 1e-6 if pid % 8 != 1 else 1e-3)
        fp = O.trace_functional(tab, 1000.0, reqs, S, G, [pid], [hstep], freeze=True)
        fm = O.trace_functional(tab, 1000.0, reqs, S, G, [pid], [-hstep], freeze=True)
        fd = (fp - fm) / (2 * hstep)
        assert grad[j] == pytest.approx(fd, rel=2e-5, abs=1e-9 * max(1.0, abs(fd))), pid
        assert abs(grad[j]) > 0


def test_trace_functional_at_zero_matches_bank():
    """The functional at delta = 0 is <G, bilinear per-ray-normalised PSF>."""
    tab = W.doublet_pair_f18()
    S = dp_sensor(0.002)
    reqs = W.bank_grid([0.4], [800.0], [W.LAMBDA_D], 32, 65)
    rng = np.random.default_rng(1)
    G = [rng.standard_normal((2, 65, 65))]
    psf, _ = O.psf_bank(tab, 1000.0, reqs, S, O.MODE_BILINEAR, O.NORM_PER_RAY)
    val = O.trace_functional(tab, 1000.0, reqs, S, G, freeze=True)
    assert val == pytest.approx(float((G[0] * psf[0]).sum()), rel=1e-12)


# --------------------------------------------------------------------------
# 2-D field points (per-pixel PSF maps): the lens is rotationally symmetric,
# so the trace must commute with rotations of the field point that map the
# square pupil grid onto itself, and with the mirror x -> -x.
# --------------------------------------------------------------------------
def _req2d(h, v, depth, lam, n, ks):
    r = np.zeros(1, dtype=W.REQ_DTYPE)
    r["h_mm"], r["v_mm"], r["depth_mm"], r["lambda_nm"] = h, v, depth, lam
    r["n_grid"], r["ks"] = n, ks
    return r


def _sorted_rows(*cols):
    a = np.stack(cols, 1)
    return a[np.lexsort(a.T[::-1])]


@pytest.mark.parametrize("lens", ["doublet", "rf50"])
def test_quarter_turn_of_field_point_rotates_hits(lens):
    """Field point (0, rho) traces the quarter-turned rays of (rho, 0): the
    cell-centred pupil grid is invariant under a quarter turn, so the hit
    sets agree as sets: (x, y, dx, dy) -> (-y, x, -dy, dx)."""
    if lens == "doublet":
        tab, focus, ps, rho = W.doublet_pair_f18(), 1000.0, 0.002, 0.9
    else:
        tab, focus, ps, rho = W.canon_rf50(), 1000.0, 36.0 / 768, 9.0
    S = dp_sensor(ps)
    a = O.trace_hits(tab, focus, _req2d(rho, 0.0, 700.0, 587.5618, 32, 21)[0], S)
    b = O.trace_hits(tab, focus, _req2d(0.0, rho, 700.0, 587.5618, 32, 21)[0], S)
    ok_a, ok_b = a["state"] == 0, b["state"] == 0
    assert ok_a.sum() == ok_b.sum() > 0
    ra = _sorted_rows(-a["y"][ok_a], a["x"][ok_a], -a["dy"][ok_a], a["dx"][ok_a])
    rb = _sorted_rows(b["x"][ok_b], b["y"][ok_b], b["dx"][ok_b], b["dy"][ok_b])
    np.testing.assert_allclose(ra, rb, rtol=0, atol=1e-9)


def test_mirrored_field_point_swaps_left_and_right():
    """Field point (-h, v) is the x-mirror of (h, v): every ray is mirrored
    exactly (the pupil grid is symmetric and the arithmetic is odd in x), so
    L(a, b) at (-h, v) = R(ks-1-a, b) at (h, v) in integer counts (Eq. 1/2:
    s changes sign under the mirror)."""
    tab, ps = W.doublet_pair_f18(), 0.002
    S = dp_sensor(ps)
    for h, v, d in [(0.6, 0.0, 950.0), (0.5, -0.3, 1050.0), (1.2, 0.7, 1000.0)]:
        reqs = np.concatenate([_req2d(h, v, d, 587.5618, 64, 31),
                               _req2d(-h, v, d, 587.5618, 64, 31)])
        (p, q), st = O.psf_bank(tab, 1000.0, reqs, S, O.MODE_HARD, O.NORM_NONE)
        assert p.sum() > 100
        np.testing.assert_array_equal(q[0], p[1][:, ::-1])
        np.testing.assert_array_equal(q[1], p[0][:, ::-1])
        np.testing.assert_array_equal(st[0], st[1][[0, 1, 3, 2, 4, 5, 6, 7]])


def test_v_zero_row_equals_axis_field_point():
    """A request with v_mm = 0 is the radial-bank request (same PSF)."""
    cfg = W.config_singlet()
    S = dp_sensor(cfg["pitch_mm"])
    r1 = W.bank_grid([0.05], [800.0], [587.5618], 64, 31)
    r2 = _req2d(0.05, 0.0, 800.0, 587.5618, 64, 31)
    (p1,), _ = O.psf_bank(cfg["lens"], 1000.0, r1, S)
    (p2,), _ = O.psf_bank(cfg["lens"], 1000.0, r2, S)
    np.testing.assert_array_equal(p1, p2)
