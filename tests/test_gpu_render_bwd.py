"""GPU render backward against the oracle's adjoint (grad of the image and of
the bank), the adjoint identities at full size, and bitwise determinism of
both gradients.  The image gradient's strip decomposition is also checked on
shapes where its folding and phases matter (one pixel, images smaller than
the kernel, fewer rows than a row block, ragged row blocks, a 1 x 1 kernel,
the largest kernel).  Tolerance: max|err| <= 1e-4 max|ref| (FP32
accumulation)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from test_gpu_render import rand_bank

pytestmark = pytest.mark.gpu

CASES = [
    # N, C, H, W, F, Z, NL, ks
    (2, 3, 37, 70, 3, 4, 3, 15),
    (1, 3, 40, 33, 2, 3, 1, 9),      # one wavelength shared by the channels
    (1, 1, 29, 41, 3, 1, 1, 5),      # single depth slice
    (1, 2, 70, 140, 4, 5, 2, 65),
    (1, 1, 36, 44, 2, 2, 1, 127),
]


def setup(case, seed):
    N, C, H, W_, F, Z, NL, ks = case
    rng = np.random.default_rng(seed)
    aif = rng.uniform(0, 1, size=(N, C, H, W_)).astype(np.float32)
    depth = rng.uniform(0.2, 4.0, size=(N, H, W_)).astype(np.float32)
    pitch = 0.002
    fh = np.linspace(0.0, 0.8 * 0.5 * np.hypot(H, W_) * pitch, F).astype(np.float32)
    dm = (W.inverse_uniform_depths(300.0, 3000.0, Z) / 1000.0).astype(np.float32)
    if Z == 1:
        dm = np.array([1.0], dtype=np.float32)
    bank = rand_bank(rng, F, Z, NL, ks).astype(np.float32)
    G = rng.standard_normal((N, 2 * C, H, W_)).astype(np.float32)
    return aif, depth, fh, dm, pitch, bank, G


@pytest.mark.parametrize("case", CASES)
def test_backward_matches_oracle(sdlib, case):
    sd = sdlib
    aif, depth, fh, dm, pitch, bank, G = setup(case, hash(case) % 2**32)
    lay = sd.BankLayout(fh, dm, bank.shape[2], bank.shape[-1], pitch)
    ga, gb = sd.dp_render_backward(torch.tensor(G, device="cuda"),
                                   torch.tensor(aif, device="cuda"),
                                   torch.tensor(depth, device="cuda"),
                                   torch.tensor(bank, device="cuda").reshape(-1), lay)
    torch.cuda.synchronize()
    ref_a, ref_b = O.render_bank_bwd(G, aif, depth, bank.astype(np.float64), fh, dm, pitch)
    got_a = ga.cpu().numpy()
    got_b = gb.cpu().numpy().reshape(ref_b.shape)
    assert np.abs(got_a - ref_a).max() <= 1e-4 * np.abs(ref_a).max()
    assert np.abs(got_b - ref_b).max() <= 1e-4 * np.abs(ref_b).max()


@pytest.mark.parametrize("img_dt,bank_dt", [(torch.bfloat16, torch.bfloat16),
                                             (torch.float32, torch.bfloat16),
                                             (torch.float16, torch.float16)])
def test_backward_low_precision_storage(sdlib, img_dt, bank_dt):
    """BF16/FP16-stored image and bank: the adjoint of the render of the
    rounded inputs, in FP32 arithmetic (same bound as FP32 storage against
    the oracle run on the rounded values)."""
    sd = sdlib
    aif, depth, fh, dm, pitch, bank, G = setup(CASES[0], 21)
    lay = sd.BankLayout(fh, dm, bank.shape[2], bank.shape[-1], pitch, dtype=bank_dt)
    a = torch.tensor(aif, device="cuda").to(img_dt)
    b = torch.tensor(bank, device="cuda").reshape(-1).to(bank_dt)
    ga, gb = sd.dp_render_backward(torch.tensor(G, device="cuda"), a,
                                   torch.tensor(depth, device="cuda"), b, lay)
    torch.cuda.synchronize()
    assert ga.dtype == torch.float32 and gb.dtype == torch.float32
    a64 = a.float().cpu().numpy().astype(np.float64)
    b64 = b.float().cpu().numpy().astype(np.float64).reshape(bank.shape)
    ref_a, ref_b = O.render_bank_bwd(G, a64, depth, b64, fh, dm, pitch)
    got_a = ga.cpu().numpy()
    got_b = gb.cpu().numpy().reshape(ref_b.shape)
    assert np.abs(got_a - ref_a).max() <= 1e-4 * np.abs(ref_a).max()
    assert np.abs(got_b - ref_b).max() <= 1e-4 * np.abs(ref_b).max()


def test_bank_gradient_deterministic_and_workspace_checked(sdlib):
    sd = sdlib
    aif, depth, fh, dm, pitch, bank, G = setup(CASES[0], 7)
    lay = sd.BankLayout(fh, dm, 3, 15, pitch)
    args = (torch.tensor(G, device="cuda"), torch.tensor(aif, device="cuda"),
            torch.tensor(depth, device="cuda"), torch.tensor(bank, device="cuda").reshape(-1))
    _, b1 = sd.dp_render_backward(*args, lay, need_aif=False)
    _, b2 = sd.dp_render_backward(*args, lay, need_aif=False)
    torch.cuda.synchronize()
    assert torch.equal(b1, b2)
    small = torch.empty(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(sd.SdError):
        sd.dp_render_backward(*args, lay, need_aif=False, workspace=small)


def test_bank_gradient_with_fewer_split_slots(sdlib):
    # the work plan splits slices with more than a block's share of tiles
    # into two chunks while split slots remain; a workspace shortened by the
    # chunk slabs leaves none (every slice one block) or a few: each result
    # matches the oracle and repeats bitwise
    sd = sdlib
    case = CASES[3]
    N, C, H, W_, F, Z, NL, ks = case
    aif, depth, fh, dm, pitch, bank, G = setup(case, 11)
    lay = sd.BankLayout(fh, dm, NL, ks, pitch)
    args = (torch.tensor(G, device="cuda"), torch.tensor(aif, device="cuda"),
            torch.tensor(depth, device="cuda"), torch.tensor(bank, device="cuda").reshape(-1))
    _, ref = O.render_bank_bwd(G, aif, depth, bank, fh, dm, pitch)
    full = sd.render_backward_workspace(lay, N, C, H, W_)
    slab = 2 * NL * 2 * ks * ks * 4            # both chunks of one split slice
    # the smallest workspace the bank gradient accepts (no split slot): the
    # calls that are refused launch nothing
    lo, hi = 0, full
    while hi - lo > 1:
        mid = (lo + hi) // 2
        try:
            sd.dp_render_backward(*args, lay, need_aif=False,
                                  workspace=torch.empty(mid, dtype=torch.uint8, device="cuda"))
            hi = mid
        except sd.SdError:
            lo = mid
    assert hi < full - 32 * slab
    for nbytes in (full, hi, hi + 3 * slab + 1024):
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        _, b1 = sd.dp_render_backward(*args, lay, need_aif=False, workspace=ws)
        _, b2 = sd.dp_render_backward(*args, lay, need_aif=False, workspace=ws)
        torch.cuda.synchronize()
        assert torch.equal(b1, b2)
        got = b1.cpu().numpy().reshape(ref.shape)
        assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()


EDGE = [
    # N, C, H, W, F, Z, NL, ks
    (1, 1, 1, 1, 2, 2, 1, 5),        # one pixel: every tap folds onto it
    (1, 2, 3, 5, 2, 3, 2, 9),        # image smaller than the kernel
    (1, 1, 7, 200, 3, 3, 1, 31),     # fewer rows than a row block, four strips
    (2, 1, 130, 17, 2, 4, 1, 65),    # narrow and tall, ragged last row block
    (1, 1, 16, 64, 2, 2, 1, 1),      # 1 x 1 kernel: a single phase
    (1, 1, 21, 300, 2, 3, 1, 127),   # largest kernel: three phases
]


@pytest.mark.parametrize("case", EDGE)
def test_image_gradient_edge_shapes(sdlib, case):
    sd = sdlib
    aif, depth, fh, dm, pitch, bank, G = setup(case, 100 + case[-1])
    lay = sd.BankLayout(fh, dm, bank.shape[2], bank.shape[-1], pitch)
    ga, _ = sd.dp_render_backward(torch.tensor(G, device="cuda"),
                                  torch.tensor(aif, device="cuda"),
                                  torch.tensor(depth, device="cuda"),
                                  torch.tensor(bank, device="cuda").reshape(-1), lay,
                                  need_bank=False)
    torch.cuda.synchronize()
    ref_a, _ = O.render_bank_bwd(G, aif, depth, bank.astype(np.float64), fh, dm, pitch)
    assert np.abs(ga.cpu().numpy() - ref_a).max() <= 1e-4 * np.abs(ref_a).max()


def test_image_gradient_needs_aligned_workspace(sdlib):
    sd = sdlib
    aif, depth, fh, dm, pitch, bank, G = setup(CASES[0], 8)
    lay = sd.BankLayout(fh, dm, 3, 15, pitch)
    args = (torch.tensor(G, device="cuda"), torch.tensor(aif, device="cuda"),
            torch.tensor(depth, device="cuda"), torch.tensor(bank, device="cuda").reshape(-1))
    n = sd.render_backward_workspace(lay, *aif.shape)
    ws = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(sd.SdError):   # too small for the image tables
        sd.dp_render_backward(*args, lay, need_bank=False, workspace=ws[:64])
    with pytest.raises(sd.SdError):   # not 256-byte aligned
        sd.dp_render_backward(*args, lay, need_bank=False, workspace=ws[8:])
    ga, _ = sd.dp_render_backward(*args, lay, need_bank=False, workspace=ws)
    torch.cuda.synchronize()
    assert torch.isfinite(ga).all()


def test_full_size_adjoint_identities(sdlib):
    """Batch of 8 RGB 512 x 512 images, the 32 x 32 x 3 bank of 65 x 65 PSFs:
    <R(I), G> = <I, dI(G)> and <R(B), G> = <B, dB(G)> (the render is linear
    in both), evaluated in FP64 from the FP32 tensors."""
    sd = sdlib
    cfg = W.config_full_forward()
    rng = np.random.default_rng(11)
    aif = torch.tensor(W.aif_pink(8, 3, 512, 512, seed=4).astype(np.float32), device="cuda")
    depth = torch.tensor(W.depth_perlin(8, 512, 512, seed=5).astype(np.float32), device="cuda")
    bank = torch.tensor(rand_bank(rng, 32, 32, 3, 65).astype(np.float32), device="cuda").reshape(-1)
    lay = sd.BankLayout(cfg["field_h_mm"], cfg["depths_mm"] / 1000.0, 3, 65, 0.004)
    G = torch.randn((8, 6, 512, 512), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    out = sd.dp_render(aif, depth, bank, lay)
    ga, gb = sd.dp_render_backward(G, aif, depth, bank, lay)
    torch.cuda.synchronize()
    lhs = (out.double() * G.double()).sum().item()
    # FP32 accumulations over 6.3 M pixels x 8450 taps: relative 1e-4
    assert (aif.double() * ga.double()).sum().item() == pytest.approx(lhs, rel=1e-4)
    assert (bank.double() * gb.double()).sum().item() == pytest.approx(lhs, rel=1e-4)
    # both gradients are bitwise reproducible
    ga2, gb2 = sd.dp_render_backward(G, aif, depth, bank, lay)
    torch.cuda.synchronize()
    assert torch.equal(ga, ga2) and torch.equal(gb, gb2)
