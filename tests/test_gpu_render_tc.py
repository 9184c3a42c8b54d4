"""The tensor-core (tcgen05) BF16 render against the FP64 oracle on the
rounded inputs (bound 8 * 2^-9 max|ref|: BF16 output rounding plus FP32
accumulation), against the CUDA-core BF16 render, on ragged tiles, on tiles
that need several passes of 8 slices, at full size, and its validation."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from test_gpu_render import rand_bank

pytestmark = pytest.mark.gpu
BOUND = 8 * 2.0 ** -9


def scene(seed, N, C, H, W_, F, Z, NL, ks, noisy_depth=False):
    rng = np.random.default_rng(seed)
    aif = rng.uniform(0, 1, size=(N, C, H, W_)).astype(np.float32)
    if noisy_depth:   # independent per-pixel depths: many slices per tile
        depth = rng.uniform(0.3, 3.0, size=(N, H, W_)).astype(np.float32)
    else:
        depth = W.depth_perlin(N, H, W_, seed=seed).astype(np.float32)
    fh = np.linspace(0.0, 0.5 * np.hypot(H, W_) * 0.002, F).astype(np.float32)
    dm = (W.inverse_uniform_depths(300.0, 3000.0, Z) / 1000.0).astype(np.float32)
    if Z == 1:
        dm = np.array([1.0], dtype=np.float32)
    bank = rand_bank(rng, F, Z, NL, ks)
    return aif, depth, fh, dm, bank


def run_tc(sd, aif, depth, fh, dm, bank):
    lay = sd.BankLayout(fh, dm, bank.shape[2], bank.shape[-1], 0.002, dtype=torch.bfloat16)
    a = torch.tensor(aif, device="cuda").to(torch.bfloat16)
    b = torch.tensor(bank, dtype=torch.float32, device="cuda").to(torch.bfloat16).reshape(-1)
    d = torch.tensor(depth, device="cuda")
    ws = torch.empty(sd.api.render_tc_workspace(lay), dtype=torch.uint8, device="cuda")
    out = sd.dp_render_tc(a, d, b, lay, workspace=ws)
    simt = sd.dp_render(a, d, b, lay)
    torch.cuda.synchronize()
    assert int(ws[:4].view(torch.int32).item()) == 0   # no completion wait gave up
    return (out.float().cpu().numpy(), simt.float().cpu().numpy(), a.float().cpu().numpy(),
            b.float().cpu().numpy().reshape(bank.shape))


CASES = [
    # N, C, H, W, F, Z, NL, ks, noisy depth
    (1, 3, 48, 40, 4, 6, 3, 31, False),
    (2, 1, 37, 29, 3, 4, 1, 15, False),     # ragged tiles in both directions
    (1, 2, 33, 70, 4, 5, 2, 65, False),
    (1, 1, 20, 24, 2, 1, 1, 9, False),      # single depth slice
    (1, 3, 32, 24, 6, 8, 3, 17, True),      # tiles with more than 8 slices
    (1, 2, 40, 50, 5, 9, 2, 65, True),      # several passes at the largest kernel
    (1, 1, 18, 17, 2, 2, 1, 1, False),      # 1 x 1 kernel
]


@pytest.mark.parametrize("case", CASES)
def test_tc_render_matches_oracle(sdlib, case):
    sd = sdlib
    *shape, noisy = case
    aif, depth, fh, dm, bank = scene(hash(case) % 2**32, *shape, noisy_depth=noisy)
    got, simt, a_r, b_r = run_tc(sd, aif, depth, fh, dm, bank)
    ref = O.render_bank(a_r, depth, b_r, fh, dm, 0.002, n_threads=8)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= BOUND * scale
    # the CUDA-core BF16 render of the same inputs: both round an FP32 sum
    assert np.abs(got - simt).max() <= 2 * BOUND * scale


def test_tc_render_full_size_sampled_and_deterministic(sdlib):
    """1024 x 1024 RGB, 32 x 32 x 3 bank of 65 x 65 PSFs, Perlin depth."""
    sd = sdlib
    cfg = W.config_full_forward()
    rng = np.random.default_rng(5)
    aif = W.aif_pink(1, 3, 1024, 1024, seed=1).astype(np.float32)
    depth = W.depth_perlin(1, 1024, 1024, seed=2).astype(np.float32)
    bank = rand_bank(rng, 32, 32, 3, 65)
    fh, dm = cfg["field_h_mm"], cfg["depths_mm"] / 1000.0
    lay = sd.BankLayout(fh, dm, 3, 65, cfg["pitch_mm"], dtype=torch.bfloat16)
    a = torch.tensor(aif, device="cuda").to(torch.bfloat16)
    d = torch.tensor(depth, device="cuda")
    b = torch.tensor(bank, dtype=torch.float32, device="cuda").to(torch.bfloat16).reshape(-1)
    ws = torch.empty(sd.api.render_tc_workspace(lay), dtype=torch.uint8, device="cuda")
    out1 = sd.dp_render_tc(a, d, b, lay, workspace=ws)
    out2 = sd.dp_render_tc(a, d, b, lay, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(out1, out2)
    assert int(ws[:4].view(torch.int32).item()) == 0
    ys = np.concatenate([[0, 0, 1023, 1023, 511], rng.integers(0, 1024, 91)])
    xs = np.concatenate([[0, 1023, 0, 1023, 512], rng.integers(0, 1024, 91)])
    pix = np.stack([np.zeros_like(ys), ys, xs], 1)
    b_r = b.float().cpu().numpy().reshape(bank.shape)
    ref = O.render_bank_pixels(a.float().cpu().numpy(), depth, b_r, fh, dm, cfg["pitch_mm"],
                               pix, n_threads=8)
    got = out1.float().cpu().numpy()[0][:, ys, xs].T
    assert np.abs(got - ref).max() <= BOUND * np.abs(ref).max()


def test_tc_render_validation(sdlib):
    sd = sdlib
    rng = np.random.default_rng(1)
    lay = sd.BankLayout([0.0, 0.1], [0.5, 2.0], 1, 67, 0.002, dtype=torch.bfloat16)
    a = torch.zeros((1, 1, 16, 16), device="cuda", dtype=torch.bfloat16)
    d = torch.ones((1, 16, 16), device="cuda")
    b = torch.zeros(2 * 2 * 2 * 67 * 67, device="cuda", dtype=torch.bfloat16)
    with pytest.raises(sd.SdError):          # ks > 65
        sd.dp_render_tc(a, d, b, lay)
    lay2 = sd.BankLayout([0.0, 0.1], [0.5, 2.0], 1, 9, 0.002, dtype=torch.bfloat16)
    with pytest.raises(ValueError):          # image must be bfloat16
        sd.dp_render_tc(a.float(), d, b[:2 * 2 * 2 * 81], lay2)
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(sd.SdError):          # workspace too small
        sd.dp_render_tc(a, d, b[:2 * 2 * 2 * 81], lay2, workspace=small)
