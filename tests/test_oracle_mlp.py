"""Pins of the oracle's DP PSF network (Sec. 3.3): an independent float64
evaluation with library linear layers, the biases-only closed form and the
normalised input coordinates."""
import numpy as np
import torch

import oracle as O


def he_net(rng, ks):
    shapes = [(512, 3)] + [(512, 512)] * 4 + [(2 * ks * ks, 512)]
    w = [rng.normal(0, np.sqrt(2.0 / s[1]), size=s) for s in shapes]
    b = [rng.normal(0, 0.05, size=s[0]) for s in shapes]
    return w, b


def test_mlp_matches_library_layers():
    rng = np.random.default_rng(0)
    ks = 7
    w, b = he_net(rng, ks)
    p = rng.uniform(-1, 1, size=(50, 3))
    h = torch.tensor(p, dtype=torch.float64)
    for l in range(5):
        h = torch.relu(torch.nn.functional.linear(h, torch.tensor(w[l]), torch.tensor(b[l])))
    o = torch.clamp(torch.nn.functional.linear(h, torch.tensor(w[5]), torch.tensor(b[5])), min=0)
    o = (o / o.sum(1, keepdim=True)).numpy().reshape(-1, 2, ks, ks)
    got = O.mlp_psf(w, b, p, ks)
    np.testing.assert_allclose(got, o, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(got.sum(axis=(1, 2, 3)), 1.0, rtol=1e-12)
    assert got.min() >= 0


def test_mlp_biases_only_closed_form():
    """Zero weights: every point predicts ReLU(b_5) / sum ReLU(b_5); an
    all-negative output layer predicts the zero PSF."""
    rng = np.random.default_rng(1)
    ks = 5
    w, b = he_net(rng, ks)
    w = [np.zeros_like(x) for x in w]
    p = rng.uniform(-1, 1, size=(4, 3))
    got = O.mlp_psf(w, b, p, ks)
    r = np.maximum(b[5], 0)
    np.testing.assert_allclose(got, np.broadcast_to((r / r.sum()).reshape(2, ks, ks), got.shape),
                               rtol=1e-14)
    b[5] = -np.abs(b[5])
    assert np.all(O.mlp_psf(w, b, p, ks) == 0)


def test_mlp_inputs_normalisation():
    H, W = 4, 6
    d = np.full((H, W), 0.5)
    d[1, 2] = 20.0
    p = O.mlp_inputs(d, 0.5, 20.0).reshape(H, W, 3)
    np.testing.assert_allclose(p[0, 0, :2], [-(W - 1) / W, -(H - 1) / H])
    np.testing.assert_allclose(p[-1, -1, :2], [(W - 1) / W, (H - 1) / H])
    np.testing.assert_allclose(p[:, :, 0].mean(), 0, atol=1e-15)
    assert p[0, 0, 2] == -1.0 and p[1, 2, 2] == 1.0
