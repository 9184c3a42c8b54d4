"""Pins of the oracle's renderer (supplement "Local DP PSF convolution") and
of its adjoint, against closed forms, library routines and brute force."""
import numpy as np
import pytest
import scipy.ndimage as ndi
import torch

import oracle as O
import workloads as W


def rand_bank(rng, F, Z, NL, ks, joint=True):
    b = rng.uniform(0.0, 1.0, size=(F, Z, NL, 2, ks, ks))
    if joint:
        b /= b.sum(axis=(3, 4, 5), keepdims=True)
    return b


def setup(rng, N=2, C=3, H=13, W_=17, F=4, Z=5, ks=5):
    aif = rng.uniform(0, 1, size=(N, C, H, W_))
    depth = rng.uniform(0.25, 3.5, size=(N, H, W_)).astype(np.float32)
    fh = np.linspace(0.0, 0.03, F).astype(np.float32)
    depths = W.inverse_uniform_depths(300.0, 3000.0, Z) / 1000.0
    return aif, depth, fh, depths.astype(np.float32), np.float32(0.002)


def test_delta_psf_returns_input():
    """L = R = delta/2 at the patch centre: L + R reproduces the AiF image."""
    rng = np.random.default_rng(0)
    aif, depth, fh, depths, pitch = setup(rng)
    ks = 7
    bank = np.zeros((4, 5, 3, 2, ks, ks))
    bank[..., 3, 3] = 0.5
    out = O.render_bank(aif, depth, bank, fh, depths, pitch)
    np.testing.assert_allclose(out[:, :3] + out[:, 3:], aif, atol=1e-15)
    np.testing.assert_allclose(out[:, :3], 0.5 * aif, atol=1e-15)


def test_constant_image_stays_constant():
    """With jointly normalised kernels a constant image renders to a constant
    L + R (each pixel's kernels sum to one after depth interpolation)."""
    rng = np.random.default_rng(1)
    aif, depth, fh, depths, pitch = setup(rng)
    bank = rand_bank(rng, 4, 5, 3, 5)
    const = np.full_like(aif, 0.37)
    out = O.render_bank(const, depth, bank, fh, depths, pitch)
    np.testing.assert_allclose(out[:, :3] + out[:, 3:], 0.37, rtol=1e-13)


def test_shift_invariant_kernel_is_library_convolution():
    """All bank slices equal: the per-pixel render is the ordinary
    convolution with replicate ('nearest') boundaries."""
    rng = np.random.default_rng(2)
    aif, depth, fh, depths, pitch = setup(rng, N=1, C=2, H=19, W_=23, ks=7)
    K = rng.uniform(0, 1, size=(2, 7, 7))
    bank = np.broadcast_to(K, (4, 5, 1, 2, 7, 7)).copy()
    out = O.render_bank(aif, depth, bank, fh, depths, pitch)
    for c in range(2):
        for side in range(2):
            ref = ndi.convolve(aif[0, c], K[side], mode="nearest")
            np.testing.assert_allclose(out[0, side * 2 + c], ref, rtol=1e-13, atol=1e-14)


def unfold_render(aif, psf_map):
    """Independent formulation of the per-pixel render with torch unfold:
    every output pixel dots its replicate-padded neighbourhood with its own
    flipped kernel (written for this test from the supplement's description)."""
    x = torch.from_numpy(aif)
    N, C, H, W_ = x.shape
    ks = psf_map.shape[-1]
    p = (ks - 1) // 2
    xp = torch.nn.functional.pad(x, (p, p, p, p), mode="replicate")
    cols = torch.nn.functional.unfold(xp, (ks, ks))            # (N, C*ks*ks, H*W)
    cols = cols.view(N, C, ks * ks, H * W_)
    k = torch.from_numpy(psf_map).flip(-1, -2).reshape(H * W_, 2, ks * ks)
    outs = []
    for side in range(2):
        w = k[:, side, :].t()                                   # (ks*ks, H*W)
        outs.append((cols * w[None, None]).sum(2).view(N, C, H, W_))
    return torch.cat(outs, 1).numpy()


def test_map_render_matches_unfold_formulation():
    rng = np.random.default_rng(3)
    N, C, H, W_, ks = 2, 3, 9, 11, 5
    aif = rng.uniform(0, 1, size=(N, C, H, W_))
    psf_map = rng.uniform(0, 1, size=(H, W_, 2, ks, ks))
    out = O.render_map(aif, psf_map)
    np.testing.assert_allclose(out, unfold_render(aif, psf_map), rtol=1e-13)


def select_bruteforce(depth, fh, depths, pitch):
    """Nearest field height and inverse-depth bracket, in float32 numpy."""
    H, W_ = depth.shape
    f32 = np.float32
    X = (np.arange(W_, dtype=f32) - f32(0.5 * (W_ - 1))) * f32(pitch)
    Y = (np.arange(H, dtype=f32) - f32(0.5 * (H - 1))) * f32(pitch)
    rho = np.sqrt((X[None, :] * X[None, :]) + (Y[:, None] * Y[:, None])).astype(f32)
    dist = np.abs(rho[..., None] - fh[None, None, :])          # float32
    f = np.argmin(dist, axis=-1)                                # ties -> lower index
    iq = (f32(1.0) / depths.astype(f32)).astype(f32)
    q = (f32(1.0) / depth).astype(f32)
    Z = len(depths)
    z0 = np.zeros((H, W_), dtype=int)
    t = np.zeros((H, W_), dtype=f32)
    for y in range(H):
        for x in range(W_):
            if q[y, x] >= iq[0]:
                z0[y, x], t[y, x] = 0, 0.0
            elif q[y, x] <= iq[-1]:
                z0[y, x], t[y, x] = Z - 2, 1.0
            else:
                j = max(j for j in range(Z - 1) if iq[j] >= q[y, x])
                z0[y, x] = j
                t[y, x] = f32(iq[j] - q[y, x]) / f32(iq[j] - iq[j + 1])
    return f, z0, t


def test_selection_matches_bruteforce():
    rng = np.random.default_rng(4)
    H, W_ = 40, 56
    depth = rng.uniform(0.2, 4.0, size=(H, W_)).astype(np.float32)
    fh = np.linspace(0.0, 0.06, 9).astype(np.float32)
    depths = (W.inverse_uniform_depths(300.0, 3000.0, 7) / 1000).astype(np.float32)
    sel = O.render_select(depth, fh, depths, 0.002)
    f, z0, t = select_bruteforce(depth, fh, depths, 0.002)
    np.testing.assert_array_equal(sel[..., 0], f)
    np.testing.assert_array_equal(sel[..., 1], z0)
    np.testing.assert_array_equal(sel[..., 2], z0 + 1)
    np.testing.assert_array_equal(sel[..., 3], t.astype(np.float64))


def test_bank_render_equals_map_render_of_selected_kernels():
    """Bank mode = map mode with each pixel's kernel built by brute-force
    selection and linear interpolation in inverse depth."""
    rng = np.random.default_rng(5)
    aif, depth, fh, depths, pitch = setup(rng, N=1, C=1, H=12, W_=15)
    bank = rand_bank(rng, 4, 5, 1, 5)
    f, z0, t = select_bruteforce(depth[0], fh, depths, pitch)
    t = t.astype(np.float64)
    kmap = ((1 - t)[..., None, None, None] * bank[f, z0, 0]
            + t[..., None, None, None] * bank[f, z0 + 1, 0])
    np.testing.assert_allclose(O.render_bank(aif, depth, bank, fh, depths, pitch),
                               O.render_map(aif, kmap), rtol=1e-13)


def test_backward_adjoint_identities():
    """The render is linear in the image and in the bank, so the backward
    must satisfy <R(I), G> = <I, dI(G)> and <R(B), G> = <B, dB(G)>."""
    rng = np.random.default_rng(6)
    aif, depth, fh, depths, pitch = setup(rng, N=2, C=3, H=11, W_=14, ks=5)
    bank = rand_bank(rng, 4, 5, 3, 5, joint=False)
    G = rng.standard_normal((2, 6, 11, 14))
    out = O.render_bank(aif, depth, bank, fh, depths, pitch)
    gi, gb = O.render_bank_bwd(G, aif, depth, bank, fh, depths, pitch)
    lhs = float((out * G).sum())
    assert float((aif * gi).sum()) == pytest.approx(lhs, rel=1e-12)
    assert float((bank * gb).sum()) == pytest.approx(lhs, rel=1e-12)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(7)
    aif, depth, fh, depths, pitch = setup(rng, N=1, C=1, H=7, W_=8, F=2, Z=3, ks=3)
    bank = rand_bank(rng, 2, 3, 1, 3)
    G = rng.standard_normal((1, 2, 7, 8))
    gi, gb = O.render_bank_bwd(G, aif, depth, bank, fh, depths, pitch)

    def loss(a, b):
        return float((O.render_bank(a, depth, b, fh, depths, pitch) * G).sum())

    for idx in [(0, 0, 0, 0), (0, 0, 3, 4), (0, 0, 6, 7), (0, 0, 0, 7)]:
        e = np.zeros_like(aif)
        e[idx] = 1e-6
        fd = (loss(aif + e, bank) - loss(aif - e, bank)) / 2e-6
        assert gi[idx] == pytest.approx(fd, rel=1e-7, abs=1e-10)
    for idx in [(0, 0, 0, 0, 1, 1), (1, 2, 0, 1, 0, 2), (0, 1, 0, 0, 2, 0)]:
        e = np.zeros_like(bank)
        e[idx] = 1e-6
        fd = (loss(aif, bank + e) - loss(aif, bank - e)) / 2e-6
        assert gb[idx] == pytest.approx(fd, rel=1e-7, abs=1e-10)
