"""The tensor-core render and its bank gradient with FP16 operands (both
operands of a tensor-core product share the 16-bit type; FP32 accumulation).

* Render: FP16 image and bank, FP16 output, against the FP64 oracle run on
  the FP16-rounded inputs.  The output rounding (relative 2^-11) dominates;
  bound max|err| <= 2^-9 max|ref| (BF16's bound 8 * 2^-9 with three more
  mantissa bits), and against the CUDA-core FP16 render of the same inputs
  twice that.  An FP32 bank is rounded to FP16 by the call.
* Bank gradient: FP16 image; depths on the bank's planes (weights 0 or 1) and
  FP16 inputs make every operand exact, so only FP32 accumulation remains
  (<= 1e-4 max|ref|); for any depths w * G is rounded to FP16 (relative
  2^-12), elementwise |err| <= 2^-11 A + 1e-4 max|ref| with A the oracle's
  adjoint of |G| and |I|.  Deterministic, error flag clear."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from test_gpu_render import rand_bank

pytestmark = pytest.mark.gpu
BOUND = 2.0 ** -9


def f16(a):
    return torch.tensor(np.asarray(a, np.float32)).to(torch.float16).float().numpy()


def scene(seed, N, C, H, W_, F, Z, NL, ks, planes=False):
    rng = np.random.default_rng(seed)
    aif = f16(rng.uniform(0, 1, size=(N, C, H, W_)))
    dm = (W.inverse_uniform_depths(300.0, 3000.0, Z) / 1000.0).astype(np.float32)
    if planes:
        depth = dm[rng.integers(0, Z, size=(N, H, W_))].astype(np.float32)
    else:
        depth = W.depth_perlin(N, H, W_, seed=seed).astype(np.float32)
    fh = np.linspace(0.0, 0.5 * np.hypot(H, W_) * 0.002, F).astype(np.float32)
    bank = rand_bank(rng, F, Z, NL, ks)
    g = f16(rng.normal(size=(N, 2 * C, H, W_)))
    return aif, depth, fh, dm, bank, g


RENDER = [
    # N, C, H, W, F, Z, NL, ks
    (1, 3, 48, 40, 4, 6, 3, 31),
    (2, 1, 37, 29, 3, 4, 1, 15),
    (1, 2, 40, 50, 5, 9, 2, 65),
]


@pytest.mark.parametrize("case", RENDER)
@pytest.mark.parametrize("bank_dt", [torch.float16, torch.float32])
def test_fp16_tc_render_matches_oracle(sdlib, case, bank_dt):
    sd = sdlib
    aif, depth, fh, dm, bank, _ = scene(hash(case) % 2**32, *case)
    NL, ks = case[6], case[7]
    lay = sd.BankLayout(fh, dm, NL, ks, 0.002, dtype=bank_dt)
    a = torch.tensor(aif, device="cuda").to(torch.float16)
    b = torch.tensor(bank, dtype=torch.float32, device="cuda").reshape(-1).to(bank_dt)
    d = torch.tensor(depth, device="cuda")
    ws = torch.empty(sd.api.render_tc_workspace(lay), dtype=torch.uint8, device="cuda")
    out = sd.dp_render_tc(a, d, b, lay, workspace=ws)
    assert out.dtype == torch.float16
    sd.sync_status(ws[:4].view(torch.int32))
    b16 = f16(bank)   # the operands the tensor cores multiply
    ref = O.render_bank(aif, depth, b16, fh, dm, 0.002, n_threads=8)
    got = out.float().cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= BOUND * scale
    if bank_dt == torch.float16:
        lay16 = sd.BankLayout(fh, dm, NL, ks, 0.002, dtype=torch.float16)
        simt = sd.dp_render(a, d, b, lay16).float().cpu().numpy()
        assert np.abs(got - simt).max() <= 2 * BOUND * scale
    # bitwise reproducible
    out2 = sd.dp_render_tc(a, d, b, lay, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)


GRAD = [
    # N, C, H, W, F, Z, NL, ks, planes
    (1, 3, 40, 70, 3, 4, 3, 31, True),
    (2, 1, 33, 45, 2, 3, 1, 65, True),
    (1, 2, 37, 64, 3, 5, 2, 15, False),
]


@pytest.mark.parametrize("case", GRAD)
def test_fp16_tc_bank_gradient_matches_oracle(sdlib, case):
    sd = sdlib
    *shape, planes = case
    aif, depth, fh, dm, bank, g = scene(hash(case) % 2**32, *shape, planes=planes)
    N, C, H, Wd, F, Z, NL, ks = shape
    lay = sd.BankLayout(fh, dm, NL, ks, 0.002, dtype=torch.float16)
    a = torch.tensor(aif, device="cuda").to(torch.float16)
    ws = torch.empty(sd.api.bank_grad_tc_workspace(lay, N, C, H, Wd), dtype=torch.uint8,
                     device="cuda")
    gt = torch.tensor(g, device="cuda")
    d = torch.tensor(depth, device="cuda")
    out1 = sd.dp_render_bank_grad_tc(gt, a, d, lay, workspace=ws)
    sd.sync_status(ws[:4].view(torch.int32))
    out2 = sd.dp_render_bank_grad_tc(gt, a, d, lay, workspace=ws)
    sd.sync_status(ws[:4].view(torch.int32))
    assert torch.equal(out1, out2)
    got = out1.cpu().numpy().astype(np.float64).reshape(bank.shape)
    _, ref = O.render_bank_bwd(g, aif, depth, bank, fh, dm, 0.002)
    scale = np.abs(ref).max()
    if planes:
        assert np.abs(got - ref).max() <= 1e-4 * scale
    else:
        _, A = O.render_bank_bwd(np.abs(g), np.abs(aif), depth, np.abs(bank), fh, dm, 0.002)
        assert np.all(np.abs(got - ref) <= 2.0 ** -11 * A + 1e-4 * scale)
