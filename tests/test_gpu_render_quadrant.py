"""Render through a first-quadrant 2-D bank (field points on a grid of
(x, y) heights, other quadrants by the PSF's flip symmetry, Sec. 5.3)
against the oracle: FP32 storage max|err| <= 1e-4 max|ref|, BF16 storage on
the rounded inputs <= 8 * 2^-9 max|ref|; odd and even image sizes (centre
row / column on an axis), one and several depth slices, ks 1 to 65; the
tensor-core render on the rounded inputs <= 8 * 2^-9 max|ref|; the render
backward (both gradients) <= 1e-4 max|ref|."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from test_gpu_render import rand_bank

pytestmark = pytest.mark.gpu


def scene(seed, N, C, H, W_, F, Z, NL, ks, pitch=0.002):
    rng = np.random.default_rng(seed)
    aif = rng.uniform(0, 1, size=(N, C, H, W_)).astype(np.float32)
    depth = W.depth_perlin(N, H, W_, seed=seed).astype(np.float32)
    # heights over the larger half-extent, so both clamping and interior
    # brackets occur on both axes
    fh = np.linspace(0.0, 0.5 * max(H, W_) * pitch, F).astype(np.float32)
    dm = (W.inverse_uniform_depths(300.0, 3000.0, Z) / 1000.0).astype(np.float32)
    if Z == 1:
        dm = np.array([1.0], dtype=np.float32)
    bank = rand_bank(rng, F * F, Z, NL, ks)
    return aif, depth, fh, dm, bank


CASES = [
    # N, C, H, W, F, Z, NL, ks
    (1, 3, 40, 37, 4, 3, 3, 31),
    (2, 1, 33, 64, 3, 1, 1, 15),
    (1, 2, 24, 25, 5, 4, 1, 65),
    (1, 1, 17, 17, 2, 2, 1, 1),
]


@pytest.mark.parametrize("case", CASES)
def test_quadrant_render_matches_oracle(sdlib, case):
    sd = sdlib
    N, C, H, Wd, F, Z, NL, ks = case
    aif, depth, fh, dm, bank = scene(hash(case) % 2**32, *case)
    lay = sd.BankLayout(fh, dm, NL, ks, 0.002, field_mode=sd.SD_FIELD_QUADRANT)
    assert lay.shape() == bank.shape
    got = sd.dp_render(torch.tensor(aif, device="cuda"), torch.tensor(depth, device="cuda"),
                       torch.tensor(bank, dtype=torch.float32, device="cuda").reshape(-1), lay)
    torch.cuda.synchronize()
    ref = O.render_bank(aif, depth, bank, fh, dm, 0.002, n_threads=8,
                        field_mode=O.FIELD_QUADRANT)
    assert np.abs(got.cpu().numpy() - ref).max() <= 1e-4 * np.abs(ref).max()
    # the radial reading of the same first column of cells is a different render
    rad = O.render_bank(aif, depth, bank[::F][:F], fh, dm, 0.002, n_threads=8)
    if F > 2 and ks > 1:
        assert np.abs(rad - ref).max() > 1e-3 * np.abs(ref).max()


def test_quadrant_render_bf16_and_full_size(sdlib):
    """512 x 512 RGB, an 8 x 8 grid of field points x 8 depths of 65 x 65
    kernels in BF16: sampled pixels (all four corners, the axes) against
    the oracle on the rounded inputs; two runs bitwise equal."""
    sd = sdlib
    H = Wd = 512
    aif, depth, fh, dm, bank = scene(11, 1, 3, H, Wd, 8, 8, 3, 65)
    lay = sd.BankLayout(fh, dm, 3, 65, 0.002, dtype=torch.bfloat16,
                        field_mode=sd.SD_FIELD_QUADRANT)
    a = torch.tensor(aif, device="cuda").to(torch.bfloat16)
    b = torch.tensor(bank, dtype=torch.float32, device="cuda").to(torch.bfloat16).reshape(-1)
    d = torch.tensor(depth, device="cuda")
    o1 = sd.dp_render(a, d, b, lay)
    o2 = sd.dp_render(a, d, b, lay)
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)
    rng = np.random.default_rng(2)
    ys = np.concatenate([[0, 0, H - 1, H - 1, 255, 256, 255, 256], rng.integers(0, H, 56)])
    xs = np.concatenate([[0, Wd - 1, 0, Wd - 1, 255, 256, 256, 255], rng.integers(0, Wd, 56)])
    pix = np.stack([np.zeros_like(ys), ys, xs], 1)
    ref = O.render_bank_pixels(a.float().cpu().numpy(), depth,
                               b.float().cpu().numpy().reshape(bank.shape), fh, dm, 0.002, pix,
                               n_threads=8, field_mode=O.FIELD_QUADRANT)
    got = o1.float().cpu().numpy()[0][:, ys, xs].T
    assert np.abs(got - ref).max() <= 8 * 2.0 ** -9 * np.abs(ref).max()


@pytest.mark.parametrize("case", [(1, 3, 40, 37, 4, 3, 3, 31), (1, 1, 33, 48, 3, 4, 1, 65)])
def test_quadrant_render_tensor_cores(sdlib, case):
    """The tensor-core render with a quadrant bank (flip classes re-laid out
    per call) against the oracle on the BF16-rounded inputs."""
    sd = sdlib
    N, C, H, Wd, F, Z, NL, ks = case
    aif, depth, fh, dm, bank = scene(hash(case) % 2**32, *case)
    lay = sd.BankLayout(fh, dm, NL, ks, 0.002, dtype=torch.bfloat16,
                        field_mode=sd.SD_FIELD_QUADRANT)
    a = torch.tensor(aif, device="cuda").to(torch.bfloat16)
    b = torch.tensor(bank, dtype=torch.float32, device="cuda").to(torch.bfloat16).reshape(-1)
    ws = torch.empty(sd.api.render_tc_workspace(lay), dtype=torch.uint8, device="cuda")
    got = sd.dp_render_tc(a, torch.tensor(depth, device="cuda"), b, lay, workspace=ws)
    torch.cuda.synchronize()
    assert int(ws[:4].view(torch.int32).item()) == 0
    ref = O.render_bank(a.float().cpu().numpy(), depth, b.float().cpu().numpy().reshape(bank.shape),
                        fh, dm, 0.002, n_threads=8, field_mode=O.FIELD_QUADRANT)
    assert np.abs(got.float().cpu().numpy() - ref).max() <= 8 * 2.0 ** -9 * np.abs(ref).max()


@pytest.mark.parametrize("case", [(1, 2, 24, 37, 3, 3, 2, 15), (2, 1, 33, 20, 4, 2, 1, 31)])
def test_quadrant_render_backward(sdlib, case):
    """The adjoint with a quadrant bank (per-key gradients folded onto the
    stored quadrant) against the oracle's adjoint: max|err| <= 1e-4 max|ref|
    for both gradients."""
    sd = sdlib
    N, C, H, Wd, F, Z, NL, ks = case
    aif, depth, fh, dm, bank = scene(hash(case) % 2**32, *case)
    rng = np.random.default_rng(1)
    g = rng.normal(size=(N, 2 * C, H, Wd)).astype(np.float32)
    lay = sd.BankLayout(fh, dm, NL, ks, 0.002, field_mode=sd.SD_FIELD_QUADRANT)
    ga, gb = sd.dp_render_backward(torch.tensor(g, device="cuda"), torch.tensor(aif, device="cuda"),
                                   torch.tensor(depth, device="cuda"),
                                   torch.tensor(bank, dtype=torch.float32, device="cuda").reshape(-1),
                                   lay)
    torch.cuda.synchronize()
    ra, rb = O.render_bank_bwd(g, aif, depth, bank, fh, dm, 0.002, field_mode=O.FIELD_QUADRANT)
    assert np.abs(ga.cpu().numpy() - ra).max() <= 1e-4 * np.abs(ra).max()
    gbn = gb.cpu().numpy().reshape(bank.shape)
    assert np.abs(gbn - rb).max() <= 1e-4 * np.abs(rb).max()


def test_quadrant_bank_invalid_mode(sdlib):
    sd = sdlib
    aif, depth, fh, dm, bank = scene(3, 1, 1, 16, 16, 2, 2, 1, 9)
    a = torch.tensor(aif, device="cuda")
    d = torch.tensor(depth, device="cuda")
    b = torch.tensor(bank, dtype=torch.float32, device="cuda").reshape(-1)
    bad = sd.BankLayout(fh, dm, 1, 9, 0.002, field_mode=7)
    with pytest.raises(sd.SdError):
        sd.dp_render(a, d, b, bad)
