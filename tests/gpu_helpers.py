"""Shared helpers of the GPU parity tests (inputs come from workloads and
expected values from the oracle only)."""
import numpy as np
import torch

import oracle as O
import workloads as W


def oracle_sensor(ps):
    return dict(ps=ps, h=W.DP_H * ps, f=W.DP_F * ps, w=W.DP_W * ps, r=W.DP_R * ps)


def gpu_bank(sd, lenses, reqs, ps, mode=0, norm=0, dtype=torch.float32, max_n=None):
    max_ks = int(reqs["ks"].max())
    max_n = int(max_n or reqs["n_grid"].max())
    dev, total, off = sd.make_requests(reqs)
    bank, stats = sd.dp_psf_trace(lenses, sd.DPSensor(ps), dev, len(reqs), total,
                                  max_ks=max_ks, max_n=max_n, mode=mode, norm=norm,
                                  dtype=dtype)
    torch.cuda.synchronize()
    return bank, stats.cpu().numpy(), off


def split(bank, reqs, off):
    b = bank.float().cpu().numpy()
    out = []
    for i, k in enumerate(reqs["ks"]):
        out.append(b[off[i]:off[i] + 2 * k * k].reshape(2, k, k).astype(np.float64))
    return out


def marginal_rays(table, focus, req, ps, tol=1e-5):
    """Rays whose oracle decision lies within tol (mm) of a boundary."""
    h = O.trace_hits(table, focus, req, oracle_sensor(ps))
    return int((h["margin"] < tol).sum()), h
