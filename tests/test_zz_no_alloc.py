"""The allocation-free render backward (for callers that may not allocate
device memory, e.g. code confined to a host framework's memory pool) gives
the same gradients as the workspace entry point, on two calls in a row, for
a radial FP32 bank, a radial BF16 bank and a first-quadrant bank (whose
per-key gradient slab must fit in the fixed array), and rejects sizes whose slice
bitmap exceeds its fixed 16 MiB device array.

Collected last on purpose: it shares one static device array across calls,
so it also has to work after every other GPU test has run."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from paper_2503_11213_gb300 import _lib as L
from paper_2503_11213_gb300 import api
from test_gpu_render import rand_bank

pytestmark = pytest.mark.gpu
SCRATCH = 16 << 20


def call_noalloc(lib, lay, G, aif, depth, bank, ga, gb):
    N, C, H, W_ = aif.shape
    c_lay = lay.c()
    return lib.sd_dp_render_backward_noalloc(
        api._ptr(G), api._ptr(aif), api._ptr(depth), api._ptr(bank), ctypes.byref(c_lay),
        N, C, H, W_, api._ptr(ga), api._ptr(gb), api._stream())


CASES = [
    # N, C, H, W, F, Z, NL, ks, bank dtype, field mode
    (2, 3, 70, 140, 4, 5, 3, 31, torch.float32, 0),
    (1, 3, 45, 77, 4, 5, 3, 21, torch.bfloat16, 0),
    (1, 2, 40, 52, 3, 4, 1, 15, torch.float32, 1),
]


@pytest.mark.parametrize("case", CASES)
def test_noalloc_matches_workspace_entry(sdlib, case):
    sd = sdlib
    lib = L.lib()
    N, C, H, W_, F, Z, NL, ks, dt, mode = case
    rng = np.random.default_rng(21 + ks)
    aif = torch.tensor(rng.uniform(0, 1, (N, C, H, W_)), dtype=torch.float32, device="cuda")
    depth = torch.tensor(rng.uniform(0.2, 4.0, (N, H, W_)), dtype=torch.float32, device="cuda")
    cells = F * F if mode == sd.SD_FIELD_QUADRANT else F
    bank = torch.tensor(rand_bank(rng, cells, Z, NL, ks), dtype=torch.float32,
                        device="cuda").reshape(-1).to(dt)
    G = torch.tensor(rng.standard_normal((N, 2 * C, H, W_)), dtype=torch.float32, device="cuda")
    fh = np.linspace(0.0, 0.5 * max(H, W_) * 0.002, F)
    dm = W.inverse_uniform_depths(300.0, 3000.0, Z) / 1000.0
    lay = sd.BankLayout(fh, dm, NL, ks, 0.002, dtype=dt, field_mode=mode)
    # the tables, the bitmap and (quadrant bank) the per-key slab must fit
    assert sd.render_backward_workspace(lay, N, C, H, W_) < SCRATCH
    ref_a, ref_b = sd.dp_render_backward(G, aif, depth, bank, lay)
    for _ in range(2):
        ga = torch.full_like(aif, 123.0)
        gb = torch.full(bank.shape, 123.0, dtype=torch.float32, device="cuda")
        assert call_noalloc(lib, lay, G, aif, depth, bank, ga, gb) == L.SD_OK
        torch.cuda.synchronize()
        assert (ga - ref_a).abs().max().item() <= 1e-4 * ref_a.abs().max().item()
        assert (gb - ref_b).abs().max().item() <= 1e-4 * ref_b.abs().max().item()


def test_noalloc_rejects_oversized_bitmap(sdlib):
    sd = sdlib
    lib = L.lib()
    # 250 x 256 slices: 2000 bitmap words per 64 x 32 tile; 60 x 80 tiles
    F, Z, ks, H, W_ = 250, 256, 1, 32 * 60, 64 * 80
    lay = sd.BankLayout(np.linspace(0.0, 1.0, F), np.linspace(0.3, 3.0, Z), 1, ks, 0.002)
    # the bitmap alone (one bit per key, whole 32-bit words, per 64 x 32
    # tile) exceeds the array by a wide margin
    bitmap = 60 * 80 * -(-F * Z // 32) * 4
    assert bitmap > 2 * SCRATCH
    aif = torch.zeros((1, 1, H, W_), device="cuda")
    depth = torch.ones((1, H, W_), device="cuda")
    bank = torch.zeros(F * Z * 2 * ks * ks, device="cuda")
    G = torch.zeros((1, 2, H, W_), device="cuda")
    ga, gb = torch.empty_like(aif), torch.empty_like(bank)
    assert call_noalloc(lib, lay, G, aif, depth, bank, ga, gb) == L.SD_ERR_CAPACITY
