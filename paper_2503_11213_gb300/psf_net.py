"""Fitting the DP PSF prediction network to ray-traced DP PSFs (Sec. 3.2,
"Pixel-wise DP image rendering module", Eq. 4; supplement, "DP PSF
prediction network").

The network maps the normalised object point p = (x_n, y_n, d_n) of a pixel
(its sensor position scaled to [-1, 1] and its depth scaled linearly from the
valid range to [-1, 1]) through 5 hidden layers of 512 ReLU neurons to the
2 ks^2 values of (PSF_L, PSF_R).  Training follows the paper:

* ground truth: DP PSFs ray-traced by this library (sd_dp_psf_trace, hard
  binning) at random points of the valid imaging region, each pair divided
  by its largest value over both planes (max normalisation);
* loss: Eq. 4, the L2 distance of the predicted and traced L plane plus that
  of the R plane (a mean over the elements here, a constant factor);
* inference: outputs clamped at 0 and sum-normalised jointly, done by the
  library's tensor-core kernel (sd_mlp_psf_map) on the packed weights.

Training is a one-off fit, off the rendering path: it runs as ordinary
PyTorch layers with autograd and Adam on the GPU, one step captured in a
CUDA graph and replayed.  Points are drawn uniformly
in the normalised coordinates of the region (the paper samples "random
points within the valid imaging region"); a pool of them is traced once and
minibatches are drawn from the pool.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import api


def sample_points(rng, n, sensor_hw, pitch_mm, d_min_m, d_max_m):
    """n random points of the valid imaging region: normalised (x_n, y_n,
    d_n) uniform in [-1, 1]^3, with the sensor positions (mm) and depths
    (mm) they stand for.  The normalisation is the one sd_mlp_psf_map uses:
    x_n = X / (W/2 pitch), y_n = Y / (H/2 pitch), d_n linear in depth."""
    H, W = sensor_hw
    p = rng.uniform(-1.0, 1.0, size=(n, 3))
    x_mm = p[:, 0] * 0.5 * W * pitch_mm
    y_mm = p[:, 1] * 0.5 * H * pitch_mm
    d_m = d_min_m + 0.5 * (p[:, 2] + 1.0) * (d_max_m - d_min_m)
    return p, x_mm, y_mm, d_m * 1000.0


def requests_at(x_mm, y_mm, depth_mm, lambda_nm, n_grid, ks):
    """One PSF request per point (2-D field point (x, y) on the sensor)."""
    reqs = np.zeros(len(x_mm), dtype=api.L.REQUEST_DTYPE)
    reqs["h_mm"], reqs["v_mm"], reqs["depth_mm"] = x_mm, y_mm, depth_mm
    reqs["lambda_nm"], reqs["n_grid"], reqs["ks"] = lambda_nm, n_grid, ks
    return reqs


def traced_psfs(lens, sensor, reqs, device, norm=api.L.SD_NORM_JOINT, chunk=65536):
    """DP PSFs (n, 2, ks, ks) FP32 of the requests, traced on the device
    (hard binning, joint sum normalisation by default)."""
    ks = int(reqs["ks"][0])
    n_grid = int(reqs["n_grid"][0])
    out = torch.empty((len(reqs), 2, ks, ks), dtype=torch.float32, device=device)
    for i in range(0, len(reqs), chunk):
        part = reqs[i:i + chunk]
        dev_req, total, _ = api.make_requests(part, device=device)
        bank, _ = api.dp_psf_trace(lens, sensor, dev_req, len(part), total, max_ks=ks,
                                   max_n=n_grid, norm=norm)
        out[i:i + len(part)] = bank.view(len(part), 2, ks, ks)
    return out


def max_normalised(psf):
    """Each pair divided by its largest value over L and R (zero pairs stay
    zero): the training target of the paper."""
    m = psf.flatten(1).amax(dim=1).clamp_min(1e-30)
    return psf / m.view(-1, 1, 1, 1)


def he_init(rng, ks):
    """He-initialised weights and zero biases of the six layers."""
    shapes = api.MLP_SHAPES(ks)
    w = [rng.normal(0.0, math.sqrt(2.0 / s[1]), size=s).astype(np.float32) for s in shapes]
    b = [np.zeros(s[0], dtype=np.float32) for s in shapes]
    return w, b


def forward(params, p):
    """The network in FP32 (training and reference): ReLU after the input and
    hidden layers, a linear output layer; raw outputs (no clamp or norm)."""
    h = p
    for l in range(5):
        h = torch.relu(torch.nn.functional.linear(h, params[2 * l], params[2 * l + 1]))
    return torch.nn.functional.linear(h, params[10], params[11])


def sum_normalised(o):
    """Inference-time output: clamped at 0, divided by the sum over L and R."""
    o = o.clamp_min(0.0)
    s = o.sum(dim=1, keepdim=True)
    return torch.where(s > 0, o / s.clamp_min(1e-30), torch.zeros_like(o))


def fit(lens, sensor, sensor_hw, pitch_mm, d_min_m, d_max_m, lambda_nm, n_grid, ks,
        iters=20000, batch=1024, pool=1 << 17, lr=1e-3, lr_end=1e-5, seed=0, device="cuda",
        log_every=0):
    """Fits the network to traced PSFs.  Returns (weights, biases, info) with
    float32 numpy arrays in the layout PsfMLP takes and info holding the
    training time, the final loss and the loss curve.  One optimisation step
    (forward, Eq. 4 loss, backward, Adam with a cosine-decayed learning rate)
    is captured once in a CUDA graph and replayed, the minibatch indices
    drawn beforehand from a seeded generator."""
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    p, x_mm, y_mm, d_mm = sample_points(rng, pool, sensor_hw, pitch_mm, d_min_m, d_max_m)
    gt = traced_psfs(lens, sensor, requests_at(x_mm, y_mm, d_mm, lambda_nm, n_grid, ks), device)
    target = max_normalised(gt).flatten(1)
    del gt
    pts = torch.tensor(p, dtype=torch.float32, device=device)
    t_trace = time.perf_counter() - t0
    w, b = he_init(rng, ks)
    params = []
    for wl, bl in zip(w, b):
        params += [torch.tensor(wl, device=device, requires_grad=True),
                   torch.tensor(bl, device=device, requires_grad=True)]
    lr_t = torch.tensor(lr, dtype=torch.float32, device=device)
    opt = torch.optim.Adam(params, lr=lr_t, capturable=True)
    gen = torch.Generator(device=device).manual_seed(seed)
    all_idx = torch.randint(0, pool, (iters, batch), device=device, generator=gen)
    idx = all_idx[0].clone()
    half = target.shape[1] // 2

    def step():
        opt.zero_grad(set_to_none=False)
        out = forward(params, pts[idx])
        tgt = target[idx]
        # Eq. 4: L2 of the L plane plus L2 of the R plane
        loss = ((out[:, :half] - tgt[:, :half]) ** 2).mean() + \
            ((out[:, half:] - tgt[:, half:]) ** 2).mean()
        loss.backward()
        opt.step()
        return loss

    prev_tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    curve = []
    try:
        # warm-up steps on a side stream (they are real steps of the fit),
        # then one step captured and replayed
        warm = min(3, iters)
        side = torch.cuda.Stream(device=device)
        side.wait_stream(torch.cuda.current_stream(device))
        with torch.cuda.stream(side):
            for it in range(warm):
                lr_t.fill_(lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * it / iters)))
                idx.copy_(all_idx[it])
                loss = step()
                if it == 0:
                    first = float(loss.item())
        torch.cuda.current_stream(device).wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            static_loss = step()
        for it in range(warm, iters):
            lr_t.fill_(lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * it / iters)))
            idx.copy_(all_idx[it])
            graph.replay()
            if log_every and (it % log_every == 0 or it == iters - 1):
                curve.append((it, float(static_loss.item())))
        final = float(static_loss.item()) if iters > warm else float(loss.item())
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev_tf32
    torch.cuda.synchronize()
    ws = [params[2 * l].detach().cpu().numpy() for l in range(6)]
    bs = [params[2 * l + 1].detach().cpu().numpy() for l in range(6)]
    info = {"trace_s": t_trace, "train_s": time.perf_counter() - t0 - t_trace,
            "first_loss": first, "final_loss": final, "curve": curve, "iters": iters,
            "batch": batch,
            "pool": pool, "seed": seed}
    return ws, bs, info


def map_errors(pred, ref):
    """Per-element errors of sum-normalised PSF maps (..., 2, ks, ks): mean
    absolute error (L1) and mean squared error (L2) over all elements, and
    the per-PSF L1 relative to the PSF's mass."""
    d = (pred.double() - ref.double()).flatten(0, -4).flatten(1)
    r = ref.double().flatten(0, -4).flatten(1)
    return {"l1": float(d.abs().mean().item()), "l2": float((d * d).mean().item()),
            "l1_rel_mean": float((d.abs().sum(1) / r.abs().sum(1).clamp_min(1e-30)).mean().item())}
