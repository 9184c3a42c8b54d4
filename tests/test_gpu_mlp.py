"""The DP PSF network (Sec. 3.2) on the tensor cores against the oracle.

* Exactness of the operand layouts: a network whose values are exact in BF16
  (layer 0 from biases only, permutation matrices, one-hot output rows) gives
  the oracle's map to FP32 rounding.
* He-initialised random networks (the paper's weights are not available), ks
  5, 21 (the paper's) and 31, ragged last tile: the oracle evaluates the
  network in FP64 on the same BF16-rounded weights; the kernel rounds the
  activations of the 5 hidden-layer inputs to BF16 (relative 2^-9 each) and
  accumulates in FP32.  Bound per pixel: max|err| <= 2^-5 max|ref| of that
  pixel, mean over pixels of max|err| / max|ref| <= 2^-7.
* Full 512 x 768 map with ks = 21 (the paper's timed size): sampled pixels,
  deterministic, status clear; the BF16 map equals the FP32 map rounded."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def bf16(a):
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy()


def he_net(rng, ks):
    shapes = [(512, 3)] + [(512, 512)] * 4 + [(2 * ks * ks, 512)]
    w = [rng.normal(0, np.sqrt(2.0 / s[1]), size=s).astype(np.float32) for s in shapes]
    b = [rng.normal(0, 0.05, size=s[0]).astype(np.float32) for s in shapes]
    return w, b


def oracle_map(w, b, depth, dmin, dmax, ks):
    # the kernel's BF16 weights of layers 1..5 (layer 0 and biases stay FP32)
    wr = [w[0]] + [bf16(x) for x in w[1:]]
    H, Wd = depth.shape
    return O.mlp_psf(wr, b, O.mlp_inputs(depth, dmin, dmax), ks).reshape(H, Wd, 2, ks, ks)


def run(sd, w, b, depth, dmin, dmax, ks):
    net = sd.PsfMLP(w, b, ks)
    m, st = sd.mlp_psf_map(net, torch.tensor(depth, device="cuda"), dmin, dmax)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return m.cpu().numpy().astype(np.float64)


def test_mlp_layouts_exact(sdlib):
    sd = sdlib
    ks = 13
    rng = np.random.default_rng(0)
    nout = 2 * ks * ks
    w = [np.zeros((512, 3), np.float32)]
    b = [(1.0 + (np.arange(512) % 64) / 64.0).astype(np.float32)]   # exact in BF16
    for _ in range(4):
        P = np.zeros((512, 512), np.float32)
        P[np.arange(512), rng.permutation(512)] = 1.0
        w.append(P)
        b.append(np.zeros(512, np.float32))
    W5 = np.zeros((nout, 512), np.float32)
    W5[np.arange(nout), rng.integers(0, 512, nout)] = 1.0
    w.append(W5)
    b.append(np.zeros(nout, np.float32))
    depth = np.full((5, 40), 1.0, np.float32)
    got = run(sd, w, b, depth, 0.5, 20.0, ks)
    ref = oracle_map(w, b, depth, 0.5, 20.0, ks)
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=0)


@pytest.mark.parametrize("ks", [5, 21, 31])
def test_mlp_random_network_matches_oracle(sdlib, ks):
    sd = sdlib
    rng = np.random.default_rng(ks)
    w, b = he_net(rng, ks)
    depth = W.depth_perlin(1, 37, 53, seed=ks, d_near_m=0.5, d_far_m=20.0)[0].astype(np.float32)
    got = run(sd, w, b, depth, 0.5, 20.0, ks)
    ref = oracle_map(w, b, depth, 0.5, 20.0, ks)
    err = np.abs(got - ref).reshape(-1, 2 * ks * ks).max(1)
    scale = np.abs(ref).reshape(-1, 2 * ks * ks).max(1)
    rel = err / scale
    print(f"ks {ks}: per-pixel max rel err: max {rel.max():.3e} mean {rel.mean():.3e}")
    assert np.all(scale > 0)
    assert rel.max() <= 2.0 ** -5 and rel.mean() <= 2.0 ** -7
    np.testing.assert_allclose(got.reshape(-1, 2 * ks * ks).sum(1), 1.0, rtol=1e-5)


def test_mlp_full_map_sampled_and_deterministic(sdlib):
    sd = sdlib
    ks, H, Wd = 21, 512, 768
    rng = np.random.default_rng(7)
    w, b = he_net(rng, ks)
    depth = W.depth_perlin(1, H, Wd, seed=8, d_near_m=0.5, d_far_m=20.0)[0].astype(np.float32)
    net = sd.PsfMLP(w, b, ks)
    d = torch.tensor(depth, device="cuda")
    m1, s1 = sd.mlp_psf_map(net, d, 0.5, 20.0)
    m2, s2 = sd.mlp_psf_map(net, d, 0.5, 20.0)
    torch.cuda.synchronize()
    assert int(s1.item()) == 0 and int(s2.item()) == 0
    assert torch.equal(m1, m2)
    ys = np.concatenate([[0, 0, H - 1, H - 1], rng.integers(0, H, 60)])
    xs = np.concatenate([[0, Wd - 1, 0, Wd - 1], rng.integers(0, Wd, 60)])
    wr = [w[0]] + [bf16(x) for x in w[1:]]
    p = O.mlp_inputs(depth, 0.5, 20.0).reshape(H, Wd, 3)[ys, xs]
    ref = O.mlp_psf(wr, b, p, ks).reshape(len(ys), -1)
    got = m1.cpu().numpy()[ys, xs].reshape(len(ys), -1).astype(np.float64)
    rel = np.abs(got - ref).max(1) / np.abs(ref).max(1)
    assert rel.max() <= 2.0 ** -5 and rel.mean() <= 2.0 ** -7


def test_mlp_validation(sdlib):
    sd = sdlib
    rng = np.random.default_rng(3)
    w, b = he_net(rng, 5)
    with pytest.raises(ValueError):
        sd.PsfMLP(w, b, 7)
    net = sd.PsfMLP(w, b, 5)
    d = torch.ones((4, 4), device="cuda")
    with pytest.raises(sd.SdError):
        sd.mlp_psf_map(net, d, 2.0, 1.0)
    with pytest.raises(sd.SdError):
        sd.mlp_psf_map(net, d, 0.5, 20.0, dtype=torch.float16)
    with pytest.raises(sd.SdError):
        n2 = sd.PsfMLP(*he_net(rng, 33), 33)


def test_mlp_bf16_map(sdlib):
    """The BF16 map is the FP32 map rounded to BF16 (nearest even)."""
    sd = sdlib
    ks = 21
    rng = np.random.default_rng(5)
    w, b = he_net(rng, ks)
    depth = W.depth_perlin(1, 40, 70, seed=5, d_near_m=0.5, d_far_m=20.0)[0].astype(np.float32)
    net = sd.PsfMLP(w, b, ks)
    d = torch.tensor(depth, device="cuda")
    m32, s1 = sd.mlp_psf_map(net, d, 0.5, 20.0)
    m16, s2 = sd.mlp_psf_map(net, d, 0.5, 20.0, dtype=torch.bfloat16)
    torch.cuda.synchronize()
    assert int(s1.item()) == 0 and int(s2.item()) == 0 and m16.dtype == torch.bfloat16
    assert torch.equal(m16, m32.to(torch.bfloat16))


def test_mlp_map_render_pipeline(sdlib):
    """The paper's render path end to end: network map, then the listing's
    per-pixel render (sd_dp_render_map), against the oracle's network and
    listing render on the same BF16-rounded weights; the bound adds the map
    bound (2^-5 of each pixel's max) to the render's FP32 accumulation."""
    sd = sdlib
    ks, H, Wd = 21, 30, 44
    rng = np.random.default_rng(9)
    w, b = he_net(rng, ks)
    depth = W.depth_perlin(1, H, Wd, seed=9, d_near_m=0.5, d_far_m=20.0)[0].astype(np.float32)
    aif = rng.uniform(0, 1, size=(1, 3, H, Wd)).astype(np.float32)
    net = sd.PsfMLP(w, b, ks)
    m, st = sd.mlp_psf_map(net, torch.tensor(depth, device="cuda"), 0.5, 20.0)
    out = sd.dp_render_map(torch.tensor(aif, device="cuda"), m)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = O.render_map(aif, oracle_map(w, b, depth, 0.5, 20.0, ks))
    assert np.abs(out.cpu().numpy() - ref).max() <= 2.0 ** -5 * np.abs(ref).max()
