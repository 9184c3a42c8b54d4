"""The seeded synthetic inputs have the shapes, ranges and structure the
input recipe states (sizes of the benchmark configurations, depth range,
1/f image spectrum, request grids and their order) and are reproducible."""
import math

import numpy as np

import workloads as W


def test_depth_perlin_range_smoothness_and_seeds():
    d = W.depth_perlin(2, 96, 128, seed=2)
    assert d.shape == (2, 96, 128)
    for m in d:                                   # each map rescaled to [0.3, 3] m
        assert m.min() == np.float64(0.3) and abs(m.max() - 3.0) < 1e-12
    # smooth: neighbouring pixels differ by a small part of the range
    assert np.abs(np.diff(d, axis=2)).max() < 0.25 * 2.7
    assert np.abs(np.diff(d, axis=1)).max() < 0.25 * 2.7
    np.testing.assert_array_equal(d, W.depth_perlin(2, 96, 128, seed=2))
    assert not np.array_equal(d, W.depth_perlin(2, 96, 128, seed=3))
    p = W.depth_perlin(1, 64, 64, seed=8, d_near_m=0.5, d_far_m=20.0)
    assert p.min() == np.float64(0.5) and abs(p.max() - 20.0) < 1e-12


def test_aif_pink_range_and_spectrum():
    a = W.aif_pink(1, 3, 256, 256, seed=1)
    assert a.shape == (1, 3, 256, 256)
    for plane in a[0]:
        assert plane.min() == 0.0 and plane.max() == 1.0
    # radially averaged amplitude spectrum falls as 1/f: log-log slope near -1
    spec = np.abs(np.fft.fft2(a[0, 0] - a[0, 0].mean()))
    fy = np.fft.fftfreq(256)[:, None]
    fx = np.fft.fftfreq(256)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    bins = np.geomspace(4 / 256, 0.4, 12)
    mids, amps = [], []
    for lo, hi in zip(bins[:-1], bins[1:]):
        sel = (f >= lo) & (f < hi)
        mids.append(math.sqrt(lo * hi))
        amps.append(spec[sel].mean())
    slope = np.polyfit(np.log(mids), np.log(amps), 1)[0]
    assert -1.3 < slope < -0.7
    np.testing.assert_array_equal(a, W.aif_pink(1, 3, 256, 256, seed=1))


def test_aif_blurred_uniform():
    a = W.aif_blurred_uniform(64, 64, seed=0)
    assert a.shape == (1, 1, 64, 64)
    assert a.min() >= 0.0 and a.max() <= 1.0
    assert abs(a.mean() - 0.5) < 0.05
    # blurring lowers the variance of U[0, 1] noise (1/12)
    assert a.var() < 1.0 / 12.0


def test_inverse_uniform_depths():
    d = W.inverse_uniform_depths(300.0, 3000.0, 32)
    assert d[0] == 300.0 and abs(d[-1] - 3000.0) < 1e-9
    inv = 1.0 / d
    np.testing.assert_allclose(np.diff(inv), np.diff(inv)[0], rtol=1e-9)
    assert np.all(np.diff(d) > 0)


def test_bank_grid_order():
    fh, dm, lam = np.array([0.0, 1.0]), np.array([500.0, 900.0, 2000.0]), np.array([460.0, 550.0])
    r = W.bank_grid(fh, dm, lam, 64, 31)
    assert len(r) == 12
    # [field][depth][wavelength]: wavelength fastest
    assert list(r["h_mm"][:6]) == [0.0] * 6 and r["h_mm"][6] == 1.0
    assert list(r["lambda_nm"][:2]) == [460.0, 550.0]
    assert list(r["depth_mm"][:6:2]) == [500.0, 900.0, 2000.0]
    assert np.all(r["n_grid"] == 64) and np.all(r["ks"] == 31)
    q = W.bank_grid_quadrant(fh, dm, lam, 64, 31)
    assert len(q) == 24
    # [x height][y height][depth][wavelength]
    assert list(q["h_mm"][:12]) == [0.0] * 12 and list(q["v_mm"][:6]) == [0.0] * 6
    assert q["v_mm"][6] == 1.0


def test_random_requests():
    r = W.random_requests(4096, seed=3)
    assert np.all((r["n_grid"] >= 32) & (r["n_grid"] <= 512))
    assert set(np.unique(r["ks"]).tolist()) == {15, 31, 65, 127}
    assert set(np.unique(r["lens"]).tolist()) == {0, 1}
    assert np.all((r["depth_mm"] >= 300.0 - 1e-9) & (r["depth_mm"] <= 3000.0 + 1e-9))
    # log-uniform N: about half the requests below the geometric mean 128
    assert 0.4 < np.mean(r["n_grid"] < 128) < 0.6
    np.testing.assert_array_equal(r, W.random_requests(4096, seed=3))


def test_flip_batch_members_are_distinct():
    a = W.aif_pink(2, 3, 32, 32, seed=4)
    d = W.depth_perlin(2, 32, 32, seed=5)
    ai, di = W.flip_batch(list(a), list(d), 16)
    assert ai.shape == (16, 3, 32, 32) and di.shape == (16, 32, 32)
    keys = {ai[i].tobytes() for i in range(16)}
    assert len(keys) == 16


def test_benchmark_configurations():
    c = W.config_full_forward()
    assert len(c["field_h_mm"]) == 32 and len(c["depths_mm"]) == 32
    assert c["ks"] == 65 and c["n_grid"] == 256 and c["sensor_hw"] == (1024, 1024)
    half_diag = 0.5 * math.hypot(1024, 1024) * c["pitch_mm"]
    assert c["field_h_mm"][0] == 0.0 and abs(c["field_h_mm"][-1] - half_diag) < 1e-12
    assert c["depths_mm"][0] == 300.0 and abs(c["depths_mm"][-1] - 3000.0) < 1e-9
    assert len(c["lambdas_nm"]) == 3
    d = W.config_differentiation()
    assert d["n_grid"] == 128 and d["batch"] == 8 and d["image_hw"] == (512, 512)
    p = W.config_precision()
    assert (len(p["field_h_mm"]), len(p["depths_mm"])) == (64, 64)
    assert p["batch"] == 16 and p["image_hw"] == (2048, 1536) and p["ks"] == 65
    s = W.config_singlet()
    assert s["ks"] == 31 and s["n_grid"] == 64 and len(s["field_h_mm"]) == 8
    r = W.config_paper_rf50()
    assert r["sensor_hw"] == (512, 768) and r["ks"] == 21 and r["n_grid"] == 64
    assert abs(r["pitch_mm"] - 0.046875) < 1e-15
