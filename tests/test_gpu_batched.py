"""Batched persistent trace of uneven requests (two lenses, N from 32 to 512,
ks in {15, 31, 65, 127}): identical to the per-request kernel (itself
checked against the oracle), capturable in a CUDA graph, and tunable."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_helpers import oracle_sensor, split

pytestmark = pytest.mark.gpu


def batch(sd, n_req, seed, two_d=False):
    lenses = [sd.Lens(W.doublet_pair_f18(), 1000.0), sd.Lens(W.spherical4(), 1000.0)]
    reqs = W.random_requests(n_req, seed=seed)
    if two_d:  # 2-D field points (per-pixel maps): rotate each field height
        phi = np.random.default_rng(seed + 100).uniform(0, 2 * np.pi, n_req)
        h = reqs["h_mm"].copy()
        reqs["h_mm"], reqs["v_mm"] = h * np.cos(phi), h * np.sin(phi)
    dev, total, off = sd.make_requests(reqs)
    return lenses, reqs, dev, total, off


@pytest.mark.parametrize("config,two_d", [(None, False), ((256, 4096, 1), False),
                                          ((1024, 65536, 1), False), ((512, 2048, 2), False),
                                          (None, True)])
def test_batched_equals_per_request_kernel(sdlib, config, two_d):
    sd = sdlib
    lenses, reqs, dev, total, off = batch(sd, 160, seed=3, two_d=two_d)
    sensor = sd.DPSensor(0.002)
    m_ref = sd.land_mask(len(reqs), 512)
    ref, ref_st = sd.dp_psf_trace(lenses, sensor, dev, len(reqs), total, max_ks=127, max_n=512,
                                  mask=m_ref)
    m_bt = sd.land_mask(len(reqs), 512)
    m_bt.fill_(-1)  # the batched trace clears the words it owns before ORing bits in
    bt = sd.BatchedTrace(lenses, sensor, dev, len(reqs), total, max_ks=127, max_n=512,
                         config=config, mask=m_bt)
    out, st = bt.run()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert torch.equal(st, ref_st)
    # the landing masks agree on every word that holds a request's rays (the
    # items' rows start anywhere in a word: their bits are ORed in)
    words = 512 * 512 // 32
    a = m_ref.view(len(reqs), words).cpu().numpy()
    b = m_bt.view(len(reqs), words).cpu().numpy()
    used = (ref_st[:, 0].cpu().numpy() + 31) // 32
    for r in range(len(reqs)):
        assert np.array_equal(a[r, :used[r]], b[r, :used[r]]), r
    for l in lenses:
        l.free()


def test_batched_against_oracle_and_graph_replay(sdlib):
    sd = sdlib
    lenses, reqs, dev, total, off = batch(sd, 64, seed=5)
    bt = sd.BatchedTrace(lenses, sd.DPSensor(0.002), dev, len(reqs), total, max_ks=127,
                         max_n=512, norm=sd.SD_NORM_NONE)
    out, st = bt.run()
    torch.cuda.synchronize()
    first = out.clone()
    # capture the batched launch in a CUDA graph and replay it
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bt.run()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bt.run()
    out.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, first)
    # a few requests against the oracle (margin-aware exact counts)
    got = split(first, reqs, off)
    tabs = [W.doublet_pair_f18(), W.spherical4()]
    stn = st.cpu().numpy()
    for i in (0, 7, 19):
        li = int(reqs["lens"][i])
        ref, ref_st = O.psf_bank(tabs[li], 1000.0, reqs[i:i + 1], oracle_sensor(0.002),
                                 norm=O.NORM_NONE)
        h = O.trace_hits(tabs[li], 1000.0, reqs[i], oracle_sensor(0.002))
        n_marg = int((h["margin"] < 1e-5).sum())
        assert np.abs(got[i] - ref[0]).sum() <= 2 * n_marg
        assert stn[i, 0] == ref_st[0, 0]
    for l in lenses:
        l.free()


def test_tuner_picks_and_caches(sdlib, tmp_path):
    sd = sdlib
    lenses, reqs, dev, total, off = batch(sd, 96, seed=7)
    bt = sd.BatchedTrace(lenses, sd.DPSensor(0.002), dev, len(reqs), total, max_ks=127,
                         max_n=512)
    cache = tmp_path / "tune.txt"
    cfg = bt.tune(cache)
    assert cfg[0] in (256, 512, 1024) and cfg[1] >= 4096 and cfg[2] in (1, 2)
    assert cache.read_text().strip()
    again = bt.tune(cache)  # served from the cache
    assert again == cfg
    ref, _ = sd.dp_psf_trace(lenses, sd.DPSensor(0.002), dev, len(reqs), total, max_ks=127,
                             max_n=512)
    out, _ = bt.run()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    for l in lenses:
        l.free()
