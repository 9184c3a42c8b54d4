"""GPU adjoint trace against the oracle's dual-number gradient (Sec. 3.1 /
Eq. 3 in bilinear form; the oracle gradient is itself pinned by central
differences in tests/test_oracle_pins.py)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_helpers import oracle_sensor

pytestmark = pytest.mark.gpu


def config3_params(tab):
    """6 curvatures, 2 conics, 8 asphere coefficients (a4..a10 of S1, S6),
    5 inner thicknesses and the sensor distance (surfaces 1..6 of the
    doublet-pair lens; surface 0 is the stop)."""
    pids = [O.param_id(s, "c") for s in range(1, 7)]
    pids += [O.param_id(1, "k"), O.param_id(6, "k")]
    pids += [O.param_id(s, a) for s in (1, 6) for a in ("a4", "a6", "a8", "a10")]
    pids += [O.param_id(s, "t") for s in range(1, 6)]
    pids += [O.param_id(6, "t")]
    return pids


def perturbed(tab, info):
    """Config-3 target lens: all curvatures +0.5 %, sensor distance +20 um."""
    t = tab.copy()
    for s in range(1, 7):
        t[s, W.COL_R] = t[s, W.COL_R] / 1.005
    t[6, W.COL_T] = info["sensor_dist"] + 0.020
    return t


def param_scales(tab, info, pids):
    """Natural scale of each parameter: its magnitude (curvatures, asphere
    coefficients), 0.1 for conics, 0.05 mm for thicknesses."""
    out = []
    for pid in pids:
        s, j = divmod(pid, 8)
        if j == 0:
            out.append(abs(1.0 / tab[s, W.COL_R]))
        elif j == 1:
            out.append(0.1)
        elif j == 7:
            out.append(0.05)
        else:
            out.append(abs(tab[s, W.COL_A4 + j - 2]))
    return np.array(out)


def smooth_G(ks, phase):
    """A smooth functional, identical on the L and R planes: L/R decisions
    that FP32 and FP64 take differently change nothing, and a splat base
    pixel that differs moves a ray's contribution continuously."""
    a = np.arange(ks)[None, :] / ks
    b = np.arange(ks)[:, None] / ks
    g = np.cos(2 * np.pi * (1.3 * a + 0.4 * b) + phase) * np.exp(-((b - 0.5) / 0.35) ** 2) + a
    return np.stack([g, g])


def test_adjoint_exact_on_smooth_functional(sdlib):
    """Strict check of the reverse sweep (Snell, normals, Newton intersection
    by the implicit function theorem, thicknesses, sensor distance), request
    by request: the per-request gradients are large and cancel in their sum,
    so each request's partial is compared with its own oracle gradient."""
    sd = sdlib
    cfg = W.config_full_forward()
    tab, ps, focus = cfg["lens"], cfg["pitch_mm"], cfg["focus_mm"]
    info = O.lens_info(tab, focus)
    reqs = W.bank_grid([0.0, 0.7, 1.3], [450.0, 1100.0], [W.LAMBDA_D, W.LAMBDA_F], 64, 65)
    G = [smooth_G(65, 0.3 * i) for i in range(len(reqs))]
    pids = config3_params(tab)
    S = oracle_sensor(ps)
    lens = sd.Lens(tab, focus)
    dev, total, off = sd.make_requests(reqs)
    g = torch.tensor(np.concatenate([x.ravel() for x in G]), dtype=torch.float32, device="cuda")
    greq, glens = sd.dp_psf_trace_backward(lens, sd.DPSensor(ps), dev, len(reqs), g, max_ks=65,
                                           max_n=64)
    torch.cuda.synchronize()
    h = param_scales(tab, info, pids)
    rel = []
    for r in range(len(reqs)):
        ref = O.trace_grad(tab, focus, reqs[r:r + 1], S, G[r:r + 1], pids) * h
        got = greq[r].cpu().numpy().reshape(-1)[pids].astype(np.float64) * h
        rel.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    rel = np.array(rel)
    print("smooth functional per-request relative error:", np.array2string(rel, precision=2))
    # most requests agree to ~1e-5; the compact near-focus PSFs to ~2e-3
    # (FP32/FP64 splat-pixel decisions of a few rays)
    assert np.median(rel) <= 1e-4
    assert rel.max() <= 5e-3
    lens.free()


@pytest.mark.parametrize("n_grid", [128])
def test_adjoint_matches_oracle(sdlib, n_grid):
    """Gradient of the config-3 loss sum (PSF - T)^2 (bilinear, per-ray
    normalised PSFs; T traced from the perturbed lens) with respect to the
    22 lens parameters: GPU adjoint vs the oracle's dual numbers, compared
    in units of each parameter's natural scale.  With this G (not equal on
    the L and R planes, sharp near focus) the few rays per thousand whose
    side or splat pixel FP32 and FP64 decide differently shift single
    requests by up to a few percent; over the 12 requests the bound is 1 %
    of the gradient norm and 2 % per component."""
    sd = sdlib
    cfg = W.config_full_forward()
    tab, ps, focus = cfg["lens"], cfg["pitch_mm"], cfg["focus_mm"]
    info = O.lens_info(tab, focus)
    reqs = W.bank_grid([0.0, 0.7, 1.3], [450.0, 1100.0], [W.LAMBDA_D, W.LAMBDA_F], n_grid, 65)
    S = oracle_sensor(ps)
    psf, _ = O.psf_bank(tab, focus, reqs, S, O.MODE_BILINEAR, O.NORM_PER_RAY, n_threads=8)
    tgt, _ = O.psf_bank(perturbed(tab, info), 0.0, reqs, S, O.MODE_BILINEAR, O.NORM_PER_RAY,
                        n_threads=8)
    G = [2.0 * (a - b) for a, b in zip(psf, tgt)]
    pids = config3_params(tab)
    ref = O.trace_grad(tab, focus, reqs, S, G, pids, n_threads=8)
    lens = sd.Lens(tab, focus)
    dev, total, off = sd.make_requests(reqs)
    g = torch.tensor(np.concatenate([x.ravel() for x in G]), dtype=torch.float32, device="cuda")
    greq, glens = sd.dp_psf_trace_backward(lens, sd.DPSensor(ps), dev, len(reqs), g, max_ks=65,
                                           max_n=n_grid)
    torch.cuda.synchronize()
    got = glens.cpu().numpy().reshape(-1)[pids].astype(np.float64)
    # per-request partials sum to the per-lens gradient
    np.testing.assert_allclose(greq.cpu().numpy().sum(0).reshape(-1)[pids], got,
                               rtol=1e-5, atol=1e-6 * np.abs(got).max())
    h = param_scales(tab, info, pids)
    gs, rs = got * h, ref * h
    print("adjoint scaled grad (oracle):", np.array2string(rs, precision=3))
    print("adjoint scaled error       :", np.array2string(gs - rs, precision=3))
    assert np.linalg.norm(gs - rs) <= 1e-2 * np.linalg.norm(rs)
    assert np.abs(gs - rs).max() <= 2e-2 * np.abs(rs).max()
    lens.free()


def test_adjoint_with_landing_mask(sdlib):
    """The landing mask written by the forward trace (hard binning) marks the
    rays that reach the sensor on the L or R sub-pixel with their landing
    pixel at most one pixel outside the patch (the oracle's landings:
    mismatches only on rays within 1e-5 mm of a decision boundary); the
    adjoint restricted to the marked
    rays gives the unmasked adjoint's per-request gradients up to the order
    of FP32 additions, the same contributing rays, fewer swept ray slots,
    and repeats bitwise."""
    sd = sdlib
    cfg = W.config_full_forward()
    tab, ps, focus = cfg["lens"], cfg["pitch_mm"], cfg["focus_mm"]
    N = 96
    reqs = np.concatenate([
        W.bank_grid([0.0, 0.9, 1.4], [400.0, 2500.0], [W.LAMBDA_D], N, 21),
        W.bank_grid([0.5, 1.4], [700.0], [W.LAMBDA_F], N, 65)])
    n = len(reqs)
    S = oracle_sensor(ps)
    lens = sd.Lens(tab, focus)
    sensor = sd.DPSensor(ps)
    dev, total, off = sd.make_requests(reqs)
    mask = sd.land_mask(n, N)
    mask.fill_(-1)  # words past a request's rays are left as they are
    sd.dp_psf_trace(lens, sensor, dev, n, total, max_ks=65, max_n=N, mask=mask)
    torch.cuda.synchronize()
    words = (N * N + 31) // 32
    m = mask.cpu().numpy().view(np.uint32).reshape(n, words)
    for r in range(n):
        h = O.trace_hits(tab, focus, reqs[r], S)
        ks = int(reqs[r]["ks"])
        # oracle sides: 0 = L, 1 = R, 2 = neither sub-pixel
        want = (h["state"] == O.R_OK) & (h["side"] != 2) & (h["a"] >= -1) & \
               (h["a"] <= ks) & (h["b"] >= -1) & (h["b"] <= ks)
        k = np.arange(len(want))
        got = ((m[r][k >> 5] >> (k & 31).astype(np.uint32)) & 1).astype(bool)
        bad = got != want
        # FP32 and FP64 decide differently only next to a boundary, and few
        # rays lie there
        assert np.all(h["margin"][bad] < 1e-5), (r, int(bad.sum()))
        assert bad.sum() <= 3 + 0.002 * len(want)
        assert 0 < got.sum() < len(want)
    rng = np.random.default_rng(5)
    g = torch.tensor(rng.standard_normal(total), dtype=torch.float32, device="cuda")
    sw0 = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    sw1 = torch.zeros((n, 2), dtype=torch.int64, device="cuda")
    g0, _ = sd.dp_psf_trace_backward(lens, sensor, dev, n, g, max_ks=65, max_n=N, swept=sw0)
    g1, _ = sd.dp_psf_trace_backward(lens, sensor, dev, n, g, max_ks=65, max_n=N, swept=sw1,
                                     mask=mask)
    g2, _ = sd.dp_psf_trace_backward(lens, sensor, dev, n, g, max_ks=65, max_n=N, mask=mask)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)
    a0, a1 = g0.cpu().numpy().reshape(n, -1), g1.cpu().numpy().reshape(n, -1)
    for r in range(n):
        assert np.abs(a1[r] - a0[r]).max() <= 1e-4 * np.abs(a0[r]).max()
    s0, s1 = sw0.cpu().numpy(), sw1.cpu().numpy()
    assert np.array_equal(s0[:, 0], s1[:, 0])
    assert s1[:, 1].sum() < s0[:, 1].sum()
    print("swept slots without / with the mask:", s0[:, 1].sum(), s1[:, 1].sum(),
          "rays with a contribution:", s0[:, 0].sum())
    lens.free()
