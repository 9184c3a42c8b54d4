"""The render's bank gradient on the tensor cores against the oracle's
adjoint (FP64).

* Depths exactly on the bank's depth planes make every pixel weight 0 or 1,
  so the kernel's BF16 operands (image, weighted gradient) are exact when the
  inputs are BF16 numbers: only FP32 accumulation remains, bound
  max|err| <= 1e-4 max|ref| (the FP32 backward's bound).
* Any depths: the weighted gradient w * G is rounded to BF16 (relative 2^-9
  per term), so elementwise |err| <= 2^-8 * A + 1e-4 max|ref|, with A the
  oracle's adjoint of |G| and |I| (the sum of the terms' magnitudes).
* Ragged tiles, one and several channels and wavelengths, ks 15 to 65, the
  quadrant bank, deterministic, error flag clear."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from test_gpu_render import rand_bank

pytestmark = pytest.mark.gpu


def bf16(a):
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy()


def scene(seed, N, C, H, W_, F, Z, NL, ks, planes, quadrant=False):
    rng = np.random.default_rng(seed)
    aif = bf16(rng.uniform(0, 1, size=(N, C, H, W_)))
    dm = (W.inverse_uniform_depths(300.0, 3000.0, Z) / 1000.0).astype(np.float32)
    if planes:   # every pixel exactly on one of the depth planes
        depth = dm[rng.integers(0, Z, size=(N, H, W_))].astype(np.float32)
    else:
        depth = W.depth_perlin(N, H, W_, seed=seed).astype(np.float32)
    fh = np.linspace(0.0, 0.5 * np.hypot(H, W_) * 0.002, F).astype(np.float32)
    cells = F * F if quadrant else F
    bank = rand_bank(rng, cells, Z, NL, ks)
    g = bf16(rng.normal(size=(N, 2 * C, H, W_)))
    return aif, depth, fh, dm, bank, g


def run(sd, aif, depth, fh, dm, bank, g, quadrant):
    NL, ks = bank.shape[2], bank.shape[-1]
    mode = sd.SD_FIELD_QUADRANT if quadrant else sd.SD_FIELD_RADIAL
    lay = sd.BankLayout(fh, dm, NL, ks, 0.002, dtype=torch.bfloat16, field_mode=mode)
    a = torch.tensor(aif, device="cuda").to(torch.bfloat16)
    N, C, H, Wd = aif.shape
    ws = torch.empty(sd.api.bank_grad_tc_workspace(lay, N, C, H, Wd), dtype=torch.uint8,
                     device="cuda")
    gt = torch.tensor(g, device="cuda")
    d = torch.tensor(depth, device="cuda")
    out1 = sd.dp_render_bank_grad_tc(gt, a, d, lay, workspace=ws)
    flag1 = int(ws[:4].view(torch.int32).item())
    out2 = sd.dp_render_bank_grad_tc(gt, a, d, lay, workspace=ws)
    torch.cuda.synchronize()
    assert flag1 == 0 and int(ws[:4].view(torch.int32).item()) == 0
    assert torch.equal(out1, out2)
    return out1.cpu().numpy().astype(np.float64)


CASES = [
    # N, C, H, W, F, Z, NL, ks, quadrant
    (1, 3, 40, 70, 4, 3, 3, 31, False),
    (2, 1, 33, 37, 3, 4, 1, 15, False),     # ragged tiles, two images
    (1, 2, 36, 64, 3, 3, 1, 65, False),     # one bank wavelength for two channels
    (1, 1, 30, 50, 3, 2, 1, 21, True),      # quadrant bank
]


@pytest.mark.parametrize("case", CASES)
def test_bank_grad_tc_exact_weights(sdlib, case):
    sd = sdlib
    *shape, quad = case
    aif, depth, fh, dm, bank, g = scene(hash(case) % 2**32, *shape, planes=True, quadrant=quad)
    got = run(sd, aif, depth, fh, dm, bank, g, quad)
    mode = O.FIELD_QUADRANT if quad else O.FIELD_RADIAL
    _, ref = O.render_bank_bwd(g, aif, depth, bank, fh, dm, 0.002, field_mode=mode)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


@pytest.mark.parametrize("case", CASES[:2] + CASES[3:])
def test_bank_grad_tc_any_depth(sdlib, case):
    sd = sdlib
    *shape, quad = case
    aif, depth, fh, dm, bank, g = scene(hash(case) % 2**32 + 1, *shape, planes=False,
                                        quadrant=quad)
    got = run(sd, aif, depth, fh, dm, bank, g, quad)
    mode = O.FIELD_QUADRANT if quad else O.FIELD_RADIAL
    _, ref = O.render_bank_bwd(g, aif, depth, bank, fh, dm, 0.002, field_mode=mode)
    _, mag = O.render_bank_bwd(np.abs(g), np.abs(aif), depth, bank, fh, dm, 0.002, field_mode=mode)
    err = np.abs(got - ref)
    print(f"any depth: max err {err.max():.3e}, max ref {np.abs(ref).max():.3e}, "
          f"max err / magnitude sum {np.max(err / np.maximum(mag, 1e-30)):.3e}")
    assert np.all(err <= 2.0 ** -8 * mag + 1e-4 * np.abs(ref).max())


def test_bank_grad_tc_full_size(sdlib):
    """1024 x 1024 RGB, the 32 x 32 x 3 bank shape at 65 x 65, Perlin depth:
    against the CUDA-core bank gradient (FP32 accumulation of the same BF16
    image; itself parity-tested against the oracle), elementwise within
    2^-8 of the magnitude sum (the CUDA-core adjoint of |G| and |I|) plus
    1e-4 max."""
    sd = sdlib
    cfg = W.config_full_forward()
    rng = np.random.default_rng(12)
    H = Wd = 1024
    aif = W.aif_pink(1, 3, H, Wd, seed=1).astype(np.float32)
    depth = W.depth_perlin(1, H, Wd, seed=2).astype(np.float32)
    bank = rand_bank(rng, 32, 32, 3, 65)
    fh, dm = cfg["field_h_mm"], cfg["depths_mm"] / 1000.0
    lay = sd.BankLayout(fh, dm, 3, 65, cfg["pitch_mm"], dtype=torch.bfloat16)
    a = torch.tensor(aif, device="cuda").to(torch.bfloat16)
    b = torch.tensor(bank, dtype=torch.float32, device="cuda").to(torch.bfloat16).reshape(-1)
    d = torch.tensor(depth, device="cuda")
    g = torch.randn((1, 6, H, Wd), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    ws = torch.empty(sd.api.bank_grad_tc_workspace(lay, 1, 3, H, Wd), dtype=torch.uint8,
                     device="cuda")
    got = sd.dp_render_bank_grad_tc(g, a, d, lay, workspace=ws).reshape(-1)
    _, ref = sd.dp_render_backward(g, a, d, b, lay, need_aif=False)
    _, mag = sd.dp_render_backward(g.abs(), a.abs(), d, b, lay, need_aif=False)
    torch.cuda.synchronize()
    assert int(ws[:4].view(torch.int32).item()) == 0
    ref, mag = ref.reshape(-1), mag.reshape(-1)
    err = (got - ref).abs()
    assert bool((err <= 2.0 ** -8 * mag + 1e-4 * ref.abs().max()).all())
