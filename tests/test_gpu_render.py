"""GPU per-pixel DP render parity against the FP64 oracle (supplement,
"Local DP PSF convolution"; bank selection linear in inverse depth).

Tolerances: FP32 storage max|err| <= 1e-4 max|ref|; BF16/FP16 storage (inputs
rounded to the storage type and given to both sides) max|err| <= 8 * 2^-9
max|ref| for BF16 and 8 * 2^-12 for FP16 (output rounding plus FP32
accumulation).
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_helpers import oracle_sensor

pytestmark = pytest.mark.gpu


def rand_bank(rng, F, Z, NL, ks):
    """PSF-like random bank: a Gaussian blob per slice with noise, jointly
    normalised (sum L + R = 1)."""
    y, x = np.mgrid[:ks, :ks] - (ks - 1) / 2
    b = np.empty((F, Z, NL, 2, ks, ks))
    for f in range(F):
        for z in range(Z):
            for l in range(NL):
                s = rng.uniform(0.5, max(1.0, ks / 4))
                cx, cy = rng.uniform(-ks / 6, ks / 6, size=2)
                g = np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s * s))
                b[f, z, l, 0] = g * (1 + 0.3 * rng.uniform(size=g.shape)) * (x >= cx)
                b[f, z, l, 1] = g * (1 + 0.3 * rng.uniform(size=g.shape)) * (x < cx)
    b /= b.sum(axis=(3, 4, 5), keepdims=True)
    return b


def run(sd, aif, depth, bank, fh, dm, pitch, dtype=torch.float32):
    lay = sd.BankLayout(fh, dm, bank.shape[2], bank.shape[-1], pitch, dtype=dtype)
    a = torch.tensor(aif, dtype=torch.float32, device="cuda").to(dtype)
    b = torch.tensor(bank, dtype=torch.float32, device="cuda").to(dtype).reshape(-1)
    d = torch.tensor(depth, dtype=torch.float32, device="cuda")
    out = sd.dp_render(a.contiguous(), d, b.contiguous(), lay)
    torch.cuda.synchronize()
    return out.float().cpu().numpy(), a.float().cpu().numpy(), \
        b.float().cpu().numpy().reshape(bank.shape)


def test_singlet_scene(sdlib):
    """64 x 64 grayscale scene, two fronto-parallel planes (0.6 m / 2.0 m),
    rendered with the oracle's traced 8 x 4 bank of the f/2 singlet."""
    sd = sdlib
    cfg = W.config_singlet()
    ps = cfg["pitch_mm"]
    reqs = W.bank_grid(cfg["field_h_mm"], cfg["depths_mm"], cfg["lambdas_nm"], 64, 31)
    psfs, _ = O.psf_bank(cfg["lens"], cfg["focus_mm"], reqs, oracle_sensor(ps))
    bank = np.stack(psfs).reshape(8, 4, 1, 2, 31, 31).astype(np.float32).astype(np.float64)
    aif = W.aif_blurred_uniform(64, 64, seed=0).astype(np.float32)
    depth = W.depth_two_planes(64, 64, 32, 0.6, 2.0).astype(np.float32)
    dm = cfg["depths_mm"] / 1000.0
    got, _, _ = run(sd, aif, depth, bank, cfg["field_h_mm"], dm, ps)
    ref = O.render_bank(aif, depth, bank, cfg["field_h_mm"], dm, ps)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


CASES = [
    # N, C, H, W, F, Z, NL, ks
    (1, 1, 37, 70, 3, 4, 1, 3),
    (2, 3, 50, 129, 4, 5, 3, 15),
    (1, 3, 33, 65, 2, 3, 1, 31),
    (1, 2, 70, 40, 5, 1, 2, 9),     # single depth slice
    (1, 1, 20, 23, 1, 2, 1, 1),     # ks = 1 (pure per-pixel gain)
    (1, 3, 96, 128, 6, 7, 3, 65),
]


@pytest.mark.parametrize("case", CASES)
def test_random_banks_fp32(sdlib, case):
    sd = sdlib
    N, C, H, W_, F, Z, NL, ks = case
    rng = np.random.default_rng(hash(case) % 2**32)
    aif = rng.uniform(0, 1, size=(N, C, H, W_)).astype(np.float32)
    # depths beyond both ends of the bank exercise the clamping
    depth = rng.uniform(0.2, 4.0, size=(N, H, W_)).astype(np.float32)
    pitch = 0.002
    half_diag = 0.5 * np.hypot(H, W_) * pitch
    fh = np.linspace(0.0, 0.8 * half_diag, F).astype(np.float32)
    dm = (W.inverse_uniform_depths(300.0, 3000.0, Z) / 1000.0).astype(np.float32)
    if Z == 1:
        dm = np.array([1.0], dtype=np.float32)
    bank = rand_bank(rng, F, Z, NL, ks).astype(np.float32).astype(np.float64)
    got, _, _ = run(sd, aif, depth, bank, fh, dm, pitch)
    ref = O.render_bank(aif, depth, bank, fh, dm, pitch, n_threads=8)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("dtype,bound", [(torch.bfloat16, 8 * 2.0 ** -9),
                                         (torch.float16, 8 * 2.0 ** -12)])
def test_low_precision_storage(sdlib, dtype, bound):
    sd = sdlib
    rng = np.random.default_rng(3)
    N, C, H, W_, F, Z, NL, ks = 1, 3, 64, 96, 4, 6, 3, 31
    aif = rng.uniform(0, 1, size=(N, C, H, W_)).astype(np.float32)
    depth = rng.uniform(0.3, 3.0, size=(N, H, W_)).astype(np.float32)
    fh = np.linspace(0.0, 0.1, F).astype(np.float32)
    dm = (W.inverse_uniform_depths(300.0, 3000.0, Z) / 1000.0).astype(np.float32)
    bank = rand_bank(rng, F, Z, NL, ks)
    got, a_rounded, b_rounded = run(sd, aif, depth, bank, fh, dm, 0.002, dtype=dtype)
    ref = O.render_bank(a_rounded, depth, b_rounded, fh, dm, 0.002, n_threads=8)
    err = np.abs(got - ref)
    assert err.max() <= bound * np.abs(ref).max()
    # and against the unrounded FP64 inputs the error stays within a few
    # storage ulps (reported, loosely bounded)
    ref64 = O.render_bank(aif, depth, bank, fh, dm, 0.002, n_threads=8)
    assert np.sqrt(((got - ref64) ** 2).mean()) <= 4 * bound * np.abs(ref64).max()


def test_max_kernel_size(sdlib):
    sd = sdlib
    rng = np.random.default_rng(4)
    N, C, H, W_, F, Z, NL, ks = 1, 1, 40, 72, 2, 2, 1, 127
    aif = rng.uniform(0, 1, size=(N, C, H, W_)).astype(np.float32)
    depth = rng.uniform(0.3, 3.0, size=(N, H, W_)).astype(np.float32)
    fh = np.array([0.0, 0.05], dtype=np.float32)
    dm = np.array([0.5, 2.0], dtype=np.float32)
    bank = rand_bank(rng, F, Z, NL, ks).astype(np.float32).astype(np.float64)
    got, _, _ = run(sd, aif, depth, bank, fh, dm, 0.002)
    ref = O.render_bank(aif, depth, bank, fh, dm, 0.002, n_threads=8)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


def test_full_size_sampled_and_deterministic(sdlib):
    """1024 x 1024 RGB, 32 x 32 x 3 bank of 65 x 65 PSFs, Perlin depth: the
    benchmarked configuration, 96 sampled pixels (corners, edges, interior)
    against the oracle; two runs are bitwise identical."""
    sd = sdlib
    cfg = W.config_full_forward()
    rng = np.random.default_rng(5)
    aif = W.aif_pink(1, 3, 1024, 1024, seed=1).astype(np.float32)
    depth = W.depth_perlin(1, 1024, 1024, seed=2).astype(np.float32)
    bank = rand_bank(rng, 32, 32, 3, 65).astype(np.float32).astype(np.float64)
    fh, dm = cfg["field_h_mm"], cfg["depths_mm"] / 1000.0
    lay = sd.BankLayout(fh, dm, 3, 65, cfg["pitch_mm"])
    a = torch.tensor(aif, device="cuda")
    d = torch.tensor(depth, device="cuda")
    b = torch.tensor(bank, dtype=torch.float32, device="cuda").reshape(-1)
    out1 = sd.dp_render(a, d, b, lay)
    out2 = sd.dp_render(a, d, b, lay)
    torch.cuda.synchronize()
    assert torch.equal(out1, out2)
    ys = np.concatenate([[0, 0, 1023, 1023, 511], rng.integers(0, 1024, 91)])
    xs = np.concatenate([[0, 1023, 0, 1023, 512], rng.integers(0, 1024, 91)])
    pix = np.stack([np.zeros_like(ys), ys, xs], 1)
    ref = O.render_bank_pixels(aif, depth, bank, fh, dm, cfg["pitch_mm"], pix, n_threads=8)
    got = out1.cpu().numpy()[0][:, ys, xs].T
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


def test_render_validation(sdlib):
    sd = sdlib
    a = torch.zeros((1, 3, 8, 8), device="cuda")
    d = torch.ones((1, 8, 8), device="cuda")
    b = torch.zeros(2 * 2 * 2 * 9, device="cuda")
    lay = sd.BankLayout([0.0, 0.01], [0.5, 1.0], 2, 3, 0.002)  # NL=2 != C=3
    with pytest.raises(sd.SdError):
        sd.dp_render(a, d, b, lay)
    lay = sd.BankLayout([0.01, 0.0], [0.5, 1.0], 1, 3, 0.002)  # not ascending
    with pytest.raises(sd.SdError):
        sd.dp_render(a, d, b[:36], lay)
