"""A mixed workload of the library's kernels on shapes that reach their edge
cases (ragged tiles and strips, folded rows, the largest kernel, split
bank slices, a quadrant bank, tensor-core passes, 16-bit maps), reduced to
a SHA-256 of each output's bytes.  Run by tests/test_gpu_checked.py in the
normal build (in process) and in the checked build (as a child process with
SDIRT_CHECKED=1, which also prints the checks' status): the two must agree
bit for bit and the checked build must record no failed check."""
import hashlib
import json
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for d in (ROOT, HERE):
    if d not in sys.path:
        sys.path.insert(0, d)

import workloads as W  # noqa: E402


def _h(t):
    return hashlib.sha256(t.detach().contiguous().cpu().numpy().tobytes()).hexdigest()


def _bank(rng, cells, Z, NL, ks):
    b = rng.uniform(0, 1, size=(cells, Z, NL, 2, ks, ks)).astype(np.float32)
    return b / b.sum(axis=(3, 4, 5), keepdims=True)


def run(sd):
    dev = torch.device("cuda", 0)
    out = {}
    rng = np.random.default_rng(2024)
    # trace with a landing mask, then the adjoint that reads it
    cfg = W.config_full_forward()
    lens = sd.Lens(cfg["lens"], cfg["focus_mm"])
    sensor = sd.DPSensor(cfg["pitch_mm"])
    reqs = np.concatenate([W.bank_grid([0.0, 1.3], [450.0, 2200.0], [W.LAMBDA_D], 64, 65),
                           W.bank_grid([0.8], [900.0], [W.LAMBDA_F], 64, 21)])
    req_dev, total, _ = sd.make_requests(reqs, device=dev)
    mask = sd.land_mask(len(reqs), 64, device=dev)
    bank, stats = sd.dp_psf_trace(lens, sensor, req_dev, len(reqs), total, max_ks=65, max_n=64,
                                  mask=mask)
    out["trace"] = _h(bank)
    g = torch.tensor(rng.standard_normal(total), dtype=torch.float32, device=dev)
    greq, _ = sd.dp_psf_trace_backward(lens, sensor, req_dev, len(reqs), g, max_ks=65, max_n=64,
                                       mask=mask)
    out["adjoint"] = _h(greq)
    lens.free()
    # bank render and its adjoint: ragged shapes, a large kernel, a quadrant bank
    for name, (N, C, H, Wd, F, Z, NL, ks, mode) in {
            "radial": (2, 3, 37, 70, 3, 4, 3, 65, 0),
            "tall": (1, 1, 130, 17, 2, 4, 1, 65, 0),
            "wide_k": (1, 1, 21, 300, 2, 3, 1, 127, 0),
            "quadrant": (1, 2, 40, 52, 3, 4, 2, 15, 1)}.items():
        cells = F * F if mode == 1 else F
        aif = torch.tensor(rng.uniform(0, 1, (N, C, H, Wd)), dtype=torch.float32, device=dev)
        depth = torch.tensor(rng.uniform(0.2, 4.0, (N, H, Wd)), dtype=torch.float32, device=dev)
        b = torch.tensor(_bank(rng, cells, Z, NL, ks), device=dev).reshape(-1)
        fh = np.linspace(0.0, 0.5 * max(H, Wd) * 0.002, F)
        dm = W.inverse_uniform_depths(300.0, 3000.0, Z) / 1000.0
        lay = sd.BankLayout(fh, dm, NL, ks, 0.002, field_mode=mode)
        o = sd.dp_render(aif, depth, b, lay)
        G = torch.tensor(rng.standard_normal(tuple(o.shape)), dtype=torch.float32, device=dev)
        ga, gb = sd.dp_render_backward(G, aif, depth, b, lay)
        out[name + "_render"] = _h(o)
        out[name + "_grad_aif"] = _h(ga)
        out[name + "_grad_bank"] = _h(gb)
        if ks <= 65:
            a16 = aif.to(torch.float16)
            lay16 = sd.BankLayout(fh, dm, NL, ks, 0.002, dtype=torch.float16, field_mode=mode)
            b16 = b.to(torch.float16)
            ws = torch.empty(sd.api.render_tc_workspace(lay16), dtype=torch.uint8, device=dev)
            out[name + "_render_tc"] = _h(sd.dp_render_tc(a16, depth, b16, lay16, workspace=ws))
            wsb = torch.empty(sd.api.bank_grad_tc_workspace(lay16, N, C, H, Wd),
                              dtype=torch.uint8, device=dev)
            out[name + "_bank_grad_tc"] = _h(sd.dp_render_bank_grad_tc(G, a16, depth, lay16,
                                                                       workspace=wsb))
    # map render, FP32 and BF16 maps
    H, Wd, ks = 24, 50, 21
    aif = torch.tensor(rng.uniform(0, 1, (1, 3, H, Wd)), dtype=torch.float32, device=dev)
    kmap = torch.tensor(rng.uniform(0, 1, (H, Wd, 2, ks, ks)), dtype=torch.float32, device=dev)
    out["map_f32"] = _h(sd.dp_render_map(aif, kmap))
    out["map_bf16"] = _h(sd.dp_render_map(aif, kmap.to(torch.bfloat16)))
    torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    import paper_2503_11213_gb300 as sd
    res = run(sd)
    site, index, bound, count = sd.api.check_status()
    print(json.dumps({"hashes": res, "site": site, "index": index, "bound": bound,
                      "count": count}))
