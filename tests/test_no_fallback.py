"""The product path has no CPU fallback: a missing CUDA library and host
tensors both fail loudly instead of computing anything on the CPU."""
import numpy as np
import pytest
import torch

import paper_2503_11213_gb300 as sd
from paper_2503_11213_gb300 import _lib as L


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "_LIB_PATH", tmp_path / "libsdirt.so")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        L.lib()


def test_host_tensors_are_refused():
    lay = sd.BankLayout(np.array([0.0, 0.5], np.float32), np.array([0.5, 2.0], np.float32), 1, 3,
                        0.004)
    aif = torch.rand(1, 1, 8, 8)
    depth = torch.full((1, 8, 8), 1.0)
    bank = torch.rand(int(np.prod(lay.shape())))
    g = torch.rand(1, 2, 8, 8)
    calls = [
        lambda: sd.dp_render(aif, depth, bank, lay),
        lambda: sd.dp_render_backward(g, aif, depth, bank, lay, need_bank=False),
        lambda: sd.dp_render_map(aif, torch.rand(8, 8, 2, 3, 3)),
    ]
    for call in calls:
        with pytest.raises((ValueError, RuntimeError)):
            call()
