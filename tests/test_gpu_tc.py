"""The tensor-core (tcgen05) path of the BF16 render on a fixed product:
descriptors, tensor-memory accumulation over two K steps and the row
window shifted through the descriptor's start address, against a float64
product of the same BF16 values."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("u", [0, 3, 8])
def test_tcgen05_product_matches(sdlib, u):
    from paper_2503_11213_gb300 import _lib as L
    from paper_2503_11213_gb300 import api
    g = torch.Generator().manual_seed(u)
    a = torch.randn((136, 32), generator=g).to(torch.bfloat16)
    b = torch.randn((16, 32), generator=g).to(torch.bfloat16)
    da, db = a.cuda(), b.cuda()
    d = torch.zeros((128, 16), device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    L.check(L.lib().sd_dev_tc_check(api._ptr(da), api._ptr(db), u, api._ptr(d), api._ptr(st),
                                    api._stream()), "sd_dev_tc_check")
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = a.double()[u:u + 128] @ b.double().T
    got = d.cpu().double()
    err = (got - ref).abs().max().item()
    print(f"u={u}: max |D - ref| = {err:.2e} (max |ref| {ref.abs().max().item():.2f})")
    assert err <= 1e-5 * ref.abs().max().item()
