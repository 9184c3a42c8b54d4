"""Pins of the first-quadrant (2-D) bank: the flip symmetry of the DP PSF
about both axes (Sec. 5.3) checked on the oracle's own trace, and the
oracle's quadrant-bank render checked against the listing render of a map of
PSFs traced at every pixel's own signed field point (no flips there)."""
import numpy as np

import oracle as O
import workloads as W
from test_oracle_pins import dp_sensor


def _req2d(h, v, depth, lam, n, ks):
    r = np.zeros(1, dtype=W.REQ_DTYPE)
    r["h_mm"], r["v_mm"], r["depth_mm"], r["lambda_nm"] = h, v, depth, lam
    r["n_grid"], r["ks"] = n, ks
    return r


def test_field_point_below_axis_mirrors_rows():
    """(h, -v) is the y-mirror of (h, v): the patch rows reverse, L and R
    stay (the DP split is along x), in integer counts."""
    tab, S = W.doublet_pair_f18(), dp_sensor(0.002)
    for h, v, d in [(0.4, 0.6, 950.0), (0.0, 0.9, 1050.0), (-0.7, 0.3, 1000.0)]:
        reqs = np.concatenate([_req2d(h, v, d, 587.5618, 64, 31),
                               _req2d(h, -v, d, 587.5618, 64, 31)])
        (p, q), st = O.psf_bank(tab, 1000.0, reqs, S, O.MODE_HARD, O.NORM_NONE)
        assert p.sum() > 100
        np.testing.assert_array_equal(q[0], p[0][::-1, :])
        np.testing.assert_array_equal(q[1], p[1][::-1, :])
        np.testing.assert_array_equal(st[0], st[1])


def _nearest(fh, r):
    """Nearest height (ties to the lower index), clamped: the renderer's rule."""
    fh = np.asarray(fh, dtype=np.float32)
    if r <= fh[0]:
        return 0
    if r >= fh[-1]:
        return len(fh) - 1
    i = int(np.searchsorted(fh, r, side="right")) - 1
    dlo, dhi = np.float32(r - fh[i]), np.float32(fh[i + 1] - r)
    return i + 1 if dhi < dlo else i


def test_quadrant_render_equals_map_of_signed_field_points():
    tab, ps, lam, depth_mm, n, ks = W.doublet_pair_f18(), 0.002, 587.5618, 980.0, 48, 9
    S = dp_sensor(ps)
    H, Wd = 7, 10                       # odd height: the centre row has Y = 0
    fh = np.array([0.0, 0.003, 0.006, 0.009], dtype=np.float32)
    F = len(fh)
    # first-quadrant bank, cell ix * F + iy at (fh[ix], fh[iy])
    qreqs = np.concatenate([_req2d(fh[ix], fh[iy], depth_mm, lam, n, ks)
                            for ix in range(F) for iy in range(F)])
    qpsf, _ = O.psf_bank(tab, 1000.0, qreqs, S)
    bank = np.stack(qpsf)[:, None, None]          # (F*F, Z=1, NL=1, 2, ks, ks)
    # every pixel's PSF traced at its own signed field point
    psf_map = np.zeros((H, Wd, 2, ks, ks))
    cache = {}
    for y in range(H):
        for x in range(Wd):
            X = (np.float32(x) - np.float32(0.5) * np.float32(Wd - 1)) * np.float32(ps)
            Y = (np.float32(y) - np.float32(0.5) * np.float32(H - 1)) * np.float32(ps)
            hx = fh[_nearest(fh, abs(X))] * (-1.0 if X < 0 else 1.0)
            hy = fh[_nearest(fh, abs(Y))] * (-1.0 if Y < 0 else 1.0)
            if (hx, hy) not in cache:
                (p,), _ = O.psf_bank(tab, 1000.0, _req2d(hx, hy, depth_mm, lam, n, ks), S)
                cache[(hx, hy)] = p
            psf_map[y, x] = cache[(hx, hy)]
    assert len(cache) > 12              # all four quadrants and both axes occur
    rng = np.random.default_rng(4)
    aif = rng.uniform(0, 1, size=(1, 2, H, Wd))
    depth = np.full((1, H, Wd), depth_mm / 1000.0, dtype=np.float32)
    ref = O.render_map(aif, psf_map)
    got = O.render_bank(aif, depth, bank, fh, np.array([depth_mm / 1000.0], np.float32), ps,
                        field_mode=O.FIELD_QUADRANT)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    # and the radial reading differs off the axes (the quadrant bank matters)
    assert not np.allclose(psf_map[0, 0], psf_map[0, -1])


def test_quadrant_render_adjoint_identity():
    """<g, render(I, B)> = <grad_I, I> and, the render being linear in the
    bank, = <grad_B, B>: the quadrant adjoint folds every flipped use back
    onto the stored element."""
    rng = np.random.default_rng(6)
    F, Z, NL, ks, H, Wd = 3, 2, 1, 5, 9, 12
    fh = np.array([0.0, 0.006, 0.012], dtype=np.float32)
    dm = np.array([0.5, 2.0], dtype=np.float32)
    bank = rng.uniform(0, 1, size=(F * F, Z, NL, 2, ks, ks))
    aif = rng.uniform(0, 1, size=(1, 2, H, Wd))
    depth = rng.uniform(0.4, 2.5, size=(1, H, Wd)).astype(np.float32)
    g = rng.normal(size=(1, 4, H, Wd))
    out = O.render_bank(aif, depth, bank, fh, dm, 0.002, field_mode=O.FIELD_QUADRANT)
    ga, gb = O.render_bank_bwd(g, aif, depth, bank, fh, dm, 0.002, field_mode=O.FIELD_QUADRANT)
    lhs = float((g * out).sum())
    np.testing.assert_allclose((ga * aif).sum(), lhs, rtol=1e-12)
    np.testing.assert_allclose((gb * bank).sum(), lhs, rtol=1e-12)
