"""Failure detection of the kernels with completion waits, without a GPU fault.

Every completion wait of the tensor-core render, its bank gradient, the
PSF network and the bulk-copy map render is a bounded poll loop; a wait that gives up sets the launch's
status word, the CTA stops issuing products, drains what it issued (a
separately bounded wait), frees its tensor memory and returns.  Here the
poll limit is set to 0 (sd_set_wait_limit), so the first wait of every CTA
gives up before any product is issued: the kernel must return, the status
word must be set, sd_sync_status must report SD_ERR_TIMEOUT, and the context
must stay usable (the same call with the default limit then succeeds and
matches a call made before the failure)."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_2503_11213_gb300 import _lib as L

pytestmark = pytest.mark.gpu


def small_scene(sd, seed=0, N=1, C=3, H=40, Wd=48, F=4, Z=5, ks=21):
    rng = np.random.default_rng(seed)
    aif = torch.tensor(rng.uniform(0, 1, size=(N, C, H, Wd)).astype(np.float32),
                       device="cuda").to(torch.bfloat16)
    depth = torch.tensor(W.depth_perlin(N, H, Wd, seed=seed).astype(np.float32), device="cuda")
    fh = np.linspace(0.0, 0.05, F).astype(np.float32)
    dm = (W.inverse_uniform_depths(300.0, 3000.0, Z) / 1000.0).astype(np.float32)
    bank = rng.uniform(0, 1, size=(F, Z, C, 2, ks, ks)).astype(np.float32)
    bank /= bank.sum(axis=(3, 4, 5), keepdims=True)
    lay = sd.BankLayout(fh, dm, C, ks, 0.002, dtype=torch.bfloat16)
    b = torch.tensor(bank, device="cuda").to(torch.bfloat16).reshape(-1)
    return aif, depth, lay, b


def expect_timeout(sd, status_word):
    with pytest.raises(sd.SdError) as e:
        sd.sync_status(status_word)
    assert e.value.status == L.SD_ERR_TIMEOUT


def test_render_tc_gives_up_and_recovers(sdlib):
    sd = sdlib
    aif, depth, lay, bank = small_scene(sd)
    ws = torch.empty(sd.api.render_tc_workspace(lay), dtype=torch.uint8, device="cuda")
    good = sd.dp_render_tc(aif, depth, bank, lay, workspace=ws)
    sd.sync_status(ws[:4].view(torch.int32))
    good = good.clone()
    out = torch.zeros_like(good)
    try:
        sd.set_wait_limit(0)
        sd.dp_render_tc(aif, depth, bank, lay, out=out, workspace=ws)
        expect_timeout(sd, ws[:4].view(torch.int32))
    finally:
        sd.set_wait_limit(None)
    again = sd.dp_render_tc(aif, depth, bank, lay, workspace=ws)
    sd.sync_status(ws[:4].view(torch.int32))
    assert torch.equal(again, good)


def test_bank_grad_tc_gives_up_and_recovers(sdlib):
    sd = sdlib
    aif, depth, lay, _ = small_scene(sd, seed=1)
    N, C, H, Wd = aif.shape
    gout = torch.randn((N, 2 * C, H, Wd), device="cuda",
                       generator=torch.Generator("cuda").manual_seed(5))
    ws = torch.empty(sd.api.bank_grad_tc_workspace(lay, N, C, H, Wd), dtype=torch.uint8,
                     device="cuda")
    good = sd.dp_render_bank_grad_tc(gout, aif, depth, lay, workspace=ws)
    sd.sync_status(ws[:4].view(torch.int32))
    good = good.clone()
    try:
        sd.set_wait_limit(0)
        sd.dp_render_bank_grad_tc(gout, aif, depth, lay, workspace=ws)
        expect_timeout(sd, ws[:4].view(torch.int32))
    finally:
        sd.set_wait_limit(None)
    again = sd.dp_render_bank_grad_tc(gout, aif, depth, lay, workspace=ws)
    sd.sync_status(ws[:4].view(torch.int32))
    assert torch.equal(again, good)


def test_mlp_gives_up_and_recovers(sdlib):
    sd = sdlib
    rng = np.random.default_rng(2)
    ks = 5
    shapes = sd.MLP_SHAPES(ks)
    net = sd.PsfMLP([rng.normal(0, np.sqrt(2.0 / s[1]), size=s).astype(np.float32)
                     for s in shapes],
                    [rng.normal(0, 0.05, size=s[0]).astype(np.float32) for s in shapes], ks)
    depth = torch.tensor(rng.uniform(0.5, 20.0, size=(19, 23)).astype(np.float32),
                         device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    good, _ = sd.mlp_psf_map(net, depth, 0.5, 20.0, status=st)
    sd.sync_status(st)
    good = good.clone()
    try:
        sd.set_wait_limit(0)
        sd.mlp_psf_map(net, depth, 0.5, 20.0, status=st)
        expect_timeout(sd, st)
    finally:
        sd.set_wait_limit(None)
    again, _ = sd.mlp_psf_map(net, depth, 0.5, 20.0, status=st)
    sd.sync_status(st)
    assert torch.equal(again, good)


def test_render_map_gives_up_and_recovers(sdlib):
    """The bulk-copy form of the map render issues its first copies before
    its first wait: with the limit at 0 that wait gives up, the warp stops,
    waits for the copies it issued and the block returns."""
    sd = sdlib
    rng = np.random.default_rng(4)
    a = torch.tensor(rng.uniform(0, 1, size=(1, 3, 24, 64)).astype(np.float32), device="cuda")
    k = torch.tensor(rng.uniform(0, 1, size=(24, 64, 2, 21, 21)).astype(np.float32),
                     device="cuda").to(torch.bfloat16)
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    good = sd.dp_render_map(a, k, status=st)
    sd.sync_status(st)
    good = good.clone()
    try:
        sd.set_wait_limit(0)
        sd.dp_render_map(a, k, status=st)
        expect_timeout(sd, st)
    finally:
        sd.set_wait_limit(None)
    again = sd.dp_render_map(a, k, status=st)
    sd.sync_status(st)
    assert torch.equal(again, good)


def test_sync_status_clear_and_null(sdlib):
    sd = sdlib
    w = torch.zeros(1, dtype=torch.int32, device="cuda")
    sd.sync_status(w)
    assert L.lib().sd_sync_status(None, None) == L.SD_ERR_ARG
