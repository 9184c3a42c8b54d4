#!/usr/bin/env python3
"""Benchmark of the DP simulator hot path on GB300.

One step = trace + bin the full PSF bank of the f/1.8 doublet-pair lens
(32 field heights x 32 depths x 3 wavelengths, 256 x 256 pupil grid, 65 x 65
L/R patches, hard binning, joint sum normalisation, FP32), render a
1024 x 1024 RGB all-in-focus image with a Perlin depth map through that bank
(FP32), back-propagate a fixed output gradient through the render to the
image and the bank (FP32), and through the trace to the lens parameters (the
adjoint trace of the bank gradient, bilinear splat, FP32).  Inputs are synthetic (workloads module) and resident in HBM before
timing; L2 is flushed (256 MiB write) before every timed step.

Prints one JSON line (rank 0).  `value` = rays traced+binned per second over
the whole step (G rays/s); the render rate and per-kernel times are extra
keys.  `--impl reference` times the FP64 CPU oracle instead on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "G rays/s traced+binned; DP Mpix/s rendered at 65x65 PSF; fwd+bwd ms vs plain"
WORKLOAD = ("doublet-pair f/1.8 lens: DP PSF bank 32 fields x 32 depths x 3 wavelengths, "
            "256x256 pupil grid, 65x65 L/R patches (hard binning, joint norm) + per-pixel "
            "DP render of 1024x1024 RGB with a Perlin depth map")
SM_COUNT_GB300 = 152
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per launch from one ncu capture of the current
# kernel, None until a capture of this build exists.  Must be re-measured
# whenever the kernel changes.
TRAFFIC_BYTES = {
    # the bank and the landing mask written (63.3 MB reached DRAM within the
    # launch), 0.7 MB read
    "trace_bin_kernel": 64.0e6,
    # every request's gradient patch read once (also the zero patches it then
    # skips) and the landing mask of the requests it traces again: 115.5 MB
    # read + 2.0 MB written; independent of the image size
    "trace_adj_kernel": 117.5e6,
    # the image-gradient call as the phase times it: selection table 4.2 MB,
    # bank re-layout 103.9 + 94.6 MB, the two strip launches 81.3 + 91.1 MB
    "render_bwd_img_kernel": 375.1e6,
    # the bank-gradient call as the phase times it: selection table 4.2 MB,
    # slice bitmap 8.4 MB, work plan 0.1 MB, bank pass 47.6 MB read + 55.3 MB
    # written (the rest of the 103.8 MB gradient bank still in L2 at its end)
    "render_bwd_bank_kernel": 115.6e6,
    # one render launch: the bank slices its tiles use and the image, 66.0 MB
    # read, 7.9 MB of output written
    "render_fwd_kernel": 73.9e6,
}

# ---------------------------------------------------------------------------
# Algorithmic FP32 work per ray (add/sub/mul/div/sqrt = 1 flop, fused
# multiply-add = 2), counted from the formulas the trace evaluates:
# ray generation (pupil sample, direction to the object point, normalise),
# per surface: conic intersection (A, B, C, discriminant, root), hit point,
# aperture test, normal, vector Snell; aspheres add Newton iterations on the
# sag (sag, its derivative, F/F' step) and the sag-gradient normal; sensor
# propagation and the Eq. 1/2 sub-pixel decision.
# ---------------------------------------------------------------------------
FLOPS_GEN = 14
FLOPS_STOP = 12
FLOPS_CONIC = 79
FLOPS_NEWTON_ITER = 50
FLOPS_ASPH_EXTRA = 15      # sag-gradient normal in place of the quadric one
NEWTON_ITERS_ASSUMED = 3
FLOPS_SENSOR_BIN = 26


# Reverse sweep of the adjoint trace per ray, counted the same way from the
# formulas trace_adj_kernel evaluates after recomputing the forward ray:
# refracting surface = sag derivatives (u, q, S1, dS1 over a4..a12), normal
# and its adjoint, Snell adjoint, implicit-intersection multiplier, transfer
# adjoint and the c, k, a4..a12 partials; the stop only has the transfer;
# sensor = propagation adjoint plus the four bilinear taps of the splat.
FLOPS_ADJ_REFRACT = 245
FLOPS_ADJ_STOP = 30
FLOPS_ADJ_SENSOR = 40


def adjoint_flops_per_ray(table):
    f = flops_per_ray(table) + FLOPS_ADJ_SENSOR
    for row in table:
        f += FLOPS_ADJ_STOP if int(row[W.COL_TYPE]) == W.SURF_STOP else FLOPS_ADJ_REFRACT
    return f


def flops_per_ray(table):
    f = FLOPS_GEN + FLOPS_SENSOR_BIN
    for row in table:
        if int(row[W.COL_TYPE]) == W.SURF_STOP:
            f += FLOPS_STOP
        else:
            f += FLOPS_CONIC
            if np.any(row[W.COL_A4:W.COL_A4 + 5] != 0):
                f += NEWTON_ITERS_ASSUMED * FLOPS_NEWTON_ITER + FLOPS_ASPH_EXTRA
    return f


def in_pupil_rays(n):
    ix = np.arange(n)
    a = 2 * ix + 1 - n
    return int(((a[:, None] ** 2 + a[None, :] ** 2) <= n * n).sum())


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""
        else:
            self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def setup_dist(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def replica_step_ms(step_ms, dist, device=None):
    """The job's step time over N replicas: the slowest rank's (max over
    ranks; every rank gets it)."""
    if not dist:
        return step_ms
    import torch
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(rays_per_step, world, step_ms):
    """Whole-job throughput in G rays/s: every replica traces its own bank
    (weak scaling, no exchange between ranks)."""
    return world * rays_per_step / (step_ms * 1e-3) / 1e9


def build_inputs(device, n_requests=0, image=0):
    """The benchmark workload; n_requests / image shrink it for profiling
    (every k-th bank request, an image x image render) -- never used for a
    reported number."""
    cfg = W.config_full_forward()
    reqs = W.bank_grid(cfg["field_h_mm"], cfg["depths_mm"], cfg["lambdas_nm"],
                       cfg["n_grid"], cfg["ks"])
    if n_requests:
        reqs = reqs[::max(1, len(reqs) // n_requests)][:n_requests]
    H, Wd = cfg["sensor_hw"]
    if image:
        H = Wd = image
    aif = W.aif_pink(1, 3, H, Wd, seed=1).astype(np.float32)
    depth = W.depth_perlin(1, H, Wd, seed=2).astype(np.float32)
    return cfg, reqs, aif, depth


def run_ours(args, world, rank, local, dist):
    import torch
    import paper_2503_11213_gb300 as sd
    from paper_2503_11213_gb300 import build as B
    B.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg, reqs, aif_np, depth_np = build_inputs(dev, args.requests, args.image)
    ps = cfg["pitch_mm"]
    sensor = sd.DPSensor(ps)
    lens = sd.Lens(cfg["lens"], cfg["focus_mm"])
    req_dev, total, off = sd.make_requests(reqs, device=dev)
    n_req = len(reqs)
    bank = torch.empty(total, dtype=torch.float32, device=dev)
    stats = torch.zeros((n_req, 8), dtype=torch.int64, device=dev)
    layout = sd.BankLayout(cfg["field_h_mm"], cfg["depths_mm"] / 1000.0, 3, cfg["ks"], ps)
    if args.requests:  # profiling subsample: a bank of the traced requests only
        layout = sd.BankLayout([0.0, 1.0], [0.3, 3.0], 3, cfg["ks"], ps)
        assert 2 * 2 * 3 * 2 * cfg["ks"] ** 2 <= total
    aif = torch.tensor(aif_np, device=dev)
    depth = torch.tensor(depth_np, device=dev)
    out = torch.empty((1, 6) + aif.shape[2:], dtype=torch.float32, device=dev)
    gout = torch.randn(out.shape, device=dev, generator=torch.Generator(dev).manual_seed(0))
    gaif = torch.empty_like(aif)
    gbank = torch.empty_like(bank)
    ws = torch.empty(max(1, sd.api.render_backward_workspace(layout, *aif.shape)),
                     dtype=torch.uint8, device=dev)
    ws_img = torch.empty_like(ws)  # the image-gradient call's own workspace
    greq = torch.empty((n_req, 32, 8), dtype=torch.float32, device=dev)
    swept = torch.zeros((n_req, 2), dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    side = torch.cuda.Stream(device=dev)
    # the forward records which rays land within a pixel of their patch; the
    # adjoint traces only those again
    mask = sd.land_mask(n_req, cfg["n_grid"], device=dev)

    def trace():
        sd.dp_psf_trace(lens, sensor, req_dev, n_req, total, max_ks=cfg["ks"],
                        max_n=cfg["n_grid"], norm=sd.SD_NORM_JOINT, out=bank, stats=stats,
                        mask=mask)

    def render():
        sd.dp_render(aif, depth, bank, layout, out=out)

    def render_bwd(img=True, bnk=True, wsp=ws):
        lay = layout.c()
        L = sd.lib()
        sd._lib.check(L.sd_dp_render_backward(
            sd.api._ptr(gout), sd.api._ptr(aif), sd.api._ptr(depth), sd.api._ptr(bank),
            sd.api.ctypes.byref(lay), 1, 3, aif.shape[2], aif.shape[3], sd.SD_F32,
            sd.api._ptr(gaif) if img else None, sd.api._ptr(gbank) if bnk else None,
            sd.api._ptr(wsp), wsp.numel(), sd.api._stream()),
            "sd_dp_render_backward")

    # the adjoint's input: the bank gradient of the render backward; in the
    # profiling subsample (a 2x2-slice render layout) that gradient is zero
    # for most requests, so a dense random gradient stands in for it there
    g_adj = gbank
    if args.requests:
        g_adj = torch.randn(gbank.shape, device=dev, generator=torch.Generator(dev).manual_seed(3))

    def trace_bwd():
        sd.dp_psf_trace_backward(lens, sensor, req_dev, n_req, g_adj, max_ks=cfg["ks"],
                                 max_n=cfg["n_grid"], norm=sd.SD_NORM_PER_RAY, grad_req=greq,
                                 swept=swept, mask=mask)

    def backward(ev=None):
        # the image-gradient call runs on a second stream beside the
        # bank-gradient call and the adjoint that reads its result (the calls
        # share no output and have separate workspaces); ev, if given,
        # receives the ends of the image call (on its stream), of the bank
        # call and of the adjoint
        fork = torch.cuda.Event()
        fork.record(stream)
        side.wait_event(fork)
        with torch.cuda.stream(side):
            render_bwd(img=True, bnk=False, wsp=ws_img)
            if ev:
                ev[0].record(side)
        render_bwd(img=False, bnk=True)
        if ev:
            ev[1].record(stream)
        trace_bwd()
        if ev:
            ev[2].record(stream)
        join = torch.cuda.Event()
        join.record(side)
        stream.wait_event(join)

    fp32 = measure_fp32_peak(sd, dev, local)

    for _ in range(args.warmup):
        trace()
        render()
        backward()
    torch.cuda.synchronize()
    rays_per_step = int(stats[:, 0].sum().item())
    # rays whose reverse sweep carries a contribution (non-zero splat
    # gradient), and the ray slots that ran it (64 per sweeping warp), in the adjoint of the step
    swept_rays = int(swept[:, 0].sum().item())
    swept_slots = int(swept[:, 1].sum().item())
    # the adjoint traces again only the requests whose gradient patch is
    # not all zero (the others have an exactly zero gradient), and of those
    # only the rays the landing mask marks
    live = g_adj.view(n_req, -1).ne(0).any(dim=1)
    live_rays = int(stats[live, 0].sum().item())
    retraced_rays = mask_rays(mask, stats[:, 0], live, n_req)

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            trace()
            ev[i][1].record(stream)
            render()
            ev[i][2].record(stream)
            backward(ev[i][3:6])
            ev[i][6].record(stream)
        # then the backward kernels alone: the same steps with the three
        # calls in sequence on one stream, for the kernels' own launch times
        # (the overlapped ones above share the GPU)
        ev_seq = [[torch.cuda.Event(enable_timing=True) for _ in range(4)]
                  for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            trace()
            render()
            ev_seq[i][0].record(stream)
            render_bwd(img=True, bnk=False, wsp=ws_img)
            ev_seq[i][1].record(stream)
            render_bwd(img=False, bnk=True)
            ev_seq[i][2].record(stream)
            trace_bwd()
            ev_seq[i][3].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()

    def phase(a, b, evs=ev):
        return [e[a].elapsed_time(e[b]) for e in evs]

    # overlapped: image gradient (on the second stream) and bank gradient
    # from the render's end, adjoint from the bank gradient's end
    t_trace, t_render = phase(0, 1), phase(1, 2)
    overlapped = {"render_bwd_img_kernel": statistics.mean(phase(2, 3)),
                  "render_bwd_bank_kernel": statistics.mean(phase(2, 4)),
                  "trace_adj_kernel": statistics.mean(phase(4, 5))}
    # alone, in sequence
    t_bimg, t_bbank, t_adj = phase(0, 1, ev_seq), phase(1, 2, ev_seq), phase(2, 3, ev_seq)
    step_ms = sum(ev[i][0].elapsed_time(ev[i][6]) for i in range(args.steps)) / args.steps
    step_ms = replica_step_ms(step_ms, dist, dev)

    # end to end through the public API: pinned host inputs in, DP image out
    h_req = torch.from_numpy(np.frombuffer(req_dev.cpu().numpy().tobytes(), np.uint8).copy()) \
        .pin_memory()
    h_aif = torch.from_numpy(aif_np).pin_memory()
    h_depth = torch.from_numpy(depth_np).pin_memory()
    h_out = torch.empty(out.shape, dtype=torch.float32).pin_memory()
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    # the image and depth uploads run on a copy stream during the trace (the
    # render waits for them), the DP image's download during the backward
    copy = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))
        e2e_ev[i][0].record(stream)
        req_dev.copy_(h_req, non_blocking=True)
        copy.wait_event(e2e_ev[i][0])  # the previous step is done with aif and depth
        with torch.cuda.stream(copy):
            aif.copy_(h_aif, non_blocking=True)
            depth.copy_(h_depth, non_blocking=True)
        inputs = torch.cuda.Event()
        inputs.record(copy)
        trace()
        stream.wait_event(inputs)
        render()
        rendered = torch.cuda.Event()
        rendered.record(stream)
        copy.wait_event(rendered)
        with torch.cuda.stream(copy):
            h_out.copy_(out, non_blocking=True)
        fetched = torch.cuda.Event()
        fetched.record(copy)
        backward()
        stream.wait_event(fetched)
        e2e_ev[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = sum(a.elapsed_time(b) for a, b in e2e_ev) / args.steps

    e2e_ms = replica_step_ms(e2e_ms, dist, dev)
    h2d = h_req.numel() + h_aif.numel() * 4 + h_depth.numel() * 4
    d2h = h_out.numel() * 4  # the DP image (gradients stay on the device)

    clocks = clk.summary()
    peaks = load_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max_mhz = peaks.get("sm_max_mhz", 2070.0)
    derived_tflops = n_sm * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    fp32_peak_tflops = fp32["tflops"] if fp32.get("tflops") else derived_tflops
    fpr = flops_per_ray(cfg["lens"])
    tr_ms = statistics.mean(t_trace)
    rd_ms = statistics.mean(t_render)
    bi_ms = statistics.mean(t_bimg)
    bb_ms = statistics.mean(t_bbank)
    bw_ms = bi_ms + bb_ms
    adj_ms = statistics.mean(t_adj)
    H, Wd = aif.shape[2:]
    # algorithmic work of each phase (FMA = 2 flops)
    render_flops = H * Wd * 3 * 2 * 2 * cfg["ks"] ** 2 * 2  # px, ch, L/R, 2 slices, FMA
    afr = adjoint_flops_per_ray(cfg["lens"])
    # the adjoint: every launched ray is traced again (the forward's work),
    # the reverse sweep counts only for the rays that carry a contribution
    adj_flops = retraced_rays * fpr + swept_rays * (afr - fpr)
    phases = {  # kernel: (flops per launch, ms per launch measured on the stream)
        "trace_bin_kernel": (rays_per_step * fpr, tr_ms),
        "render_fwd_kernel": (render_flops, rd_ms),
        # image and bank gradients: the forward's products once each
        "render_bwd_img_kernel": (render_flops, bi_ms),
        "render_bwd_bank_kernel": (render_flops, bb_ms),
        "trace_adj_kernel": (adj_flops, adj_ms),
    }
    tflops = {k: f / (ms * 1e-3) / 1e12 for k, (f, ms) in phases.items()}
    dominant = max(phases, key=lambda k: phases[k][1])
    achieved = tflops[dominant]

    def overlap_fields(k):
        if k not in overlapped:
            return {}
        tf = phases[k][0] / (overlapped[k] * 1e-3) / 1e12
        return {"ms_overlapped": round(overlapped[k], 4), "tflops_overlapped": round(tf, 3)}
    value = replica_value(rays_per_step, world, step_ms)
    e2e_value = replica_value(rays_per_step, world, e2e_ms)
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "G rays/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(step_ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rays_per_step": rays_per_step,
                   "requests": n_req, "image": [1, 3, int(H), int(Wd)],
                   "l2": "flushed before every step (256 MiB write), flush untimed",
                   "parallelism": f"replica x{world}"},
        "trace_ms": round(tr_ms, 4), "render_ms": round(rd_ms, 4),
        "render_bwd_ms": round(bw_ms, 4),
        "render_bwd_img_ms": round(bi_ms, 4), "render_bwd_bank_ms": round(bb_ms, 4),
        "render_fwd_bwd_ms": round(rd_ms + bw_ms, 4),
        "trace_adjoint_ms": round(adj_ms, 4),
        # from the render's end to the end of both streams' backward work
        "backward_span_ms": round(statistics.mean(phase(2, 6)), 4),
        "trace_grays_s": round(rays_per_step / (tr_ms * 1e-3) / 1e9, 4),
        "render_mpix_s": round(H * Wd / (rd_ms * 1e-3) / 1e6, 2),
        "roofline": {"bound": "alu", "kernel": dominant, "achieved": round(achieved, 3),
                     "peak": round(fp32_peak_tflops, 2), "unit": "TFLOP/s",
                     "frac": round(achieved / fp32_peak_tflops, 4),
                     "traffic": TRAFFIC_BYTES.get(dominant),
                     "timing": "each kernel's launch alone; in the steps that give "
                               "`value` the image-gradient call runs on a second stream "
                               "beside the bank-gradient call and the adjoint, so those "
                               "three are timed a second time, in sequence, within the same "
                               "timed region (their overlapped durations: "
                               "kernels.*.ms_overlapped)",
                     "peak_source": ("measured: FMA-chain probe on this GPU in this run, "
                                     "median of its timed launches" if fp32.get("tflops") else
                                     f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 "
                                     f"x {sm_max_mhz:.0f} MHz (max SM clock)"),
                     "fp32_probe": fp32,
                     "derived_peak_at_max_clock": round(derived_tflops, 2),
                     "flops_per_ray": fpr, "adjoint_flops_per_ray": afr,
                     "adjoint_live_request_rays": live_rays,
                     "adjoint_retraced_rays": retraced_rays,
                     "adjoint_swept_rays": swept_rays, "adjoint_swept_slots": swept_slots,
                     "adjoint_flops": adj_flops,
                     "render_flops": render_flops,
                     "kernels": {k: {"ms": round(phases[k][1], 4), "tflops": round(v, 3),
                                     "frac": round(v / fp32_peak_tflops, 4),
                                     "traffic": TRAFFIC_BYTES.get(k), **overlap_fields(k)}
                                 for k, v in tflops.items()}},
        "e2e": {"value": round(e2e_value, 4), "unit": "G rays/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": round(e2e_ms, 4)},
        # per step: trace; render; image gradient call (selection table,
        # bank re-layout, two strip phases); bank gradient call (selection
        # table, slice bitmap, slice counts, slice order, bank pass); adjoint
        # trace and lens reduce -- 13, once in the overlapped steps and once
        # in the sequential ones
        "gpu_launches": 26 * args.steps,
        "clocks": clocks,
        "wall_s": round(t_wall, 3),
    }
    if rank == 0 and not args.no_batched:
        line["uneven_batch"] = batched_compare(sd, dev)
    if rank == 0 and not args.no_extra:
        line["differentiation_pipeline"] = pipeline_compare(sd, dev)
        line["precision"] = precision_compare(sd, dev)
        line["paper_workload"] = paper_workload(sd, dev)
        line["quadrant_bank"] = quadrant_compare(sd, dev)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, reqs, aif_np, depth_np, args.cpu_seconds)
    lens.free()
    return line


def mask_rays(mask, launched, live, n_req):
    """Set bits of a landing mask over the requests in `live`, counting only
    each request's words that hold its launched rays."""
    words = mask.numel() // max(n_req, 1)
    m = mask[:n_req * words].view(n_req, words).cpu().numpy().view(np.uint32)
    nw = (launched.cpu().numpy() + 31) // 32
    keep = np.arange(words)[None, :] < nw[:, None]
    keep &= live.cpu().numpy()[:, None]
    return int(np.unpackbits(np.where(keep, m, 0).view(np.uint8)).sum())


def measure_fp32_peak(sd, dev, index, reps=40):
    """FP32 peak of this GPU: the library's FMA-chain probe (8 blocks of 256
    threads per SM, 16 independent chains per thread) timed with CUDA events,
    clocks sampled while it runs.  TFLOP/s = median over the timed launches;
    flops per SM clock from the median SM clock seen."""
    import torch
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = 8 * n_sm, 1 << 15
    sink = torch.empty(blocks * 256, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        flops = sd.fp32_peak_launch(sink, blocks, iters)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(reps)]
    with ClockSampler(index) as clk:
        for a, b in ev:
            a.record(stream)
            sd.fp32_peak_launch(sink, blocks, iters)
            b.record(stream)
        torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b) for a, b in ev)
    med = statistics.median(ms)
    c = clk.summary()
    res = {"tflops": round(flops / (med * 1e-3) / 1e12, 3),
           "tflops_best": round(flops / (ms[0] * 1e-3) / 1e12, 3),
           "ms_per_launch": round(med, 4), "flops_per_launch": flops, "launches": reps,
           "sm_mhz": c["sm_mhz"], "clock_reasons": c["reasons"]}
    if c["sm_mhz"]:
        res["flops_per_sm_clock"] = round(flops / (med * 1e-3) / (c["sm_mhz"] * 1e6) / n_sm, 2)
    return res


def batched_compare(sd, dev, reps=5):
    """Uneven requests (4096: N log-uniform 32..512, ks in {15,31,65,127},
    random field/depth/wavelength, two lenses): the batched persistent launch
    (autotuned, replayed from a CUDA graph) against one launch with one block
    per request and against one launch per request (4096 launches, also
    replayed from a graph)."""
    import ctypes
    import torch
    from paper_2503_11213_gb300 import _lib as L
    from paper_2503_11213_gb300 import api
    lenses = [sd.Lens(W.doublet_pair_f18(), 1000.0), sd.Lens(W.spherical4(), 1000.0)]
    reqs = W.random_requests(4096, seed=3)
    req_dev, total, off = sd.make_requests(reqs, device=dev)
    n_req = len(reqs)
    sensor = sd.DPSensor(0.002)
    bt = sd.BatchedTrace(lenses, sensor, req_dev, n_req, total, max_ks=127, max_n=512)
    cfg = bt.tune(os.path.join(ROOT, "paper_2503_11213_gb300", "_build", "tune_cache.txt"))
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    def graph_of(fn):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            fn()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    g_batched = graph_of(bt.run)
    t_batched = timed(g_batched.replay)
    out_plain = torch.empty(total, device=dev)
    st_plain = torch.zeros((n_req, 8), dtype=torch.int64, device=dev)

    def plain():
        sd.dp_psf_trace(lenses, sensor, req_dev, n_req, total, max_ks=127, max_n=512,
                        out=out_plain, stats=st_plain)

    t_plain = timed(plain)
    handles = (ctypes.c_void_p * 2)(*[l.handle.value for l in lenses])
    sen = sensor.c()
    lib = L.lib()
    base_req, base_out, base_st = req_dev.data_ptr(), out_plain.data_ptr(), st_plain.data_ptr()
    ks = reqs["ks"].astype(int)
    ns = reqs["n_grid"].astype(int)

    def per_request():
        for i in range(n_req):
            o = L.SdTraceOpts(0, L.SD_NORM_JOINT, 0, 0, int(ks[i]), int(ns[i]))
            L.check(lib.sd_dp_psf_trace(handles, 2, ctypes.byref(sen),
                                        ctypes.c_void_p(base_req + L.REQUEST_DTYPE.itemsize * i), 1, ctypes.byref(o),
                                        ctypes.c_void_p(base_out), ctypes.c_void_p(base_st + 64 * i),
                                        api._stream()), "sd_dp_psf_trace")

    g_per = graph_of(per_request)
    t_per = timed(g_per.replay)
    out_b, _ = bt.run()
    torch.cuda.synchronize()
    rays = int(bt.stats[:, 0].sum().item())
    same = bool(torch.equal(out_b, out_plain))
    for l in lenses:
        l.free()
    return {"requests": n_req, "rays": rays, "batched_graph_ms": round(t_batched, 4),
            "one_block_per_request_ms": round(t_plain, 4),
            "one_launch_per_request_graph_ms": round(t_per, 4),
            "batched_grays_s": round(rays / (t_batched * 1e-3) / 1e9, 3),
            "speedup_vs_per_request_launches": round(t_per / t_batched, 3),
            "speedup_vs_one_block_per_request": round(t_plain / t_batched, 3),
            "tuned_config": {"threads": cfg[0], "rays_per_item": cfg[1], "blocks_per_sm": cfg[2]},
            "identical_results": same}


def _timed(fn, stream, reps=5):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def precision_compare(sd, dev, crop=256):
    """Render a batch of 16 RGB 2048x1536 images through a 64x64x3 bank of
    65x65 PSFs stored in FP32, BF16 and FP16 (FP32 accumulation); time each
    and report its error on a crop x crop corner of image 0 (all channels,
    L and R) against the FP64 oracle render of the FP32 image and bank."""
    import torch
    import oracle as O
    c = W.config_precision()
    H, Wd = c["image_hw"]
    a_b = W.aif_pink(2, 3, H, Wd, seed=4).astype(np.float32)
    d_b = W.depth_perlin(2, H, Wd, seed=5).astype(np.float32)
    aif_np, depth_np = W.flip_batch(a_b, d_b, c["batch"])
    reqs = W.bank_grid(c["field_h_mm"], c["depths_mm"], c["lambdas_nm"], c["n_grid"], c["ks"])
    lens = sd.Lens(c["lens"], c["focus_mm"])
    sensor = sd.DPSensor(c["pitch_mm"])
    req_dev, total, _ = sd.make_requests(reqs, device=dev)
    depth = torch.tensor(depth_np, device=dev)
    aif32 = torch.tensor(aif_np, device=dev)
    stream = torch.cuda.current_stream()
    px = int(c["batch"] * H * Wd)
    res = {"batch": [c["batch"], 3, H, Wd], "bank": [64, 64, 3, 65, 65],
           "crop": f"image 0, rows/cols 0..{crop - 1}, 3 channels x L/R vs the FP64 oracle "
                   f"render of the FP32 image and FP32 bank"}
    bank32 = None
    ref = None
    fh, dm = c["field_h_mm"], c["depths_mm"] / 1000.0
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16), ("f16", torch.float16)):
        bank, _ = sd.dp_psf_trace(lens, sensor, req_dev, len(reqs), total, max_ks=c["ks"],
                                  max_n=c["n_grid"], norm=sd.SD_NORM_JOINT, dtype=dt)
        lay = sd.BankLayout(fh, dm, 3, c["ks"], c["pitch_mm"], dtype=dt)
        aif = aif32 if dt == torch.float32 else aif32.to(dt)
        out = torch.empty((c["batch"], 6, H, Wd), dtype=dt, device=dev)
        t = _timed(lambda: sd.dp_render(aif, depth, bank, lay, out=out), stream, reps=3)
        if bank32 is None:
            bank32 = bank.cpu().numpy().reshape(64, 64, 3, 2, c["ks"], c["ks"])
            ys, xs = np.meshgrid(np.arange(crop), np.arange(crop), indexing="ij")
            pix = np.stack([np.zeros(crop * crop, int), ys.ravel(), xs.ravel()], 1)
            ref = O.render_bank_pixels(aif_np[:1].astype(np.float64), depth_np[:1], bank32,
                                       fh, dm, c["pitch_mm"], pix, n_threads=cpu_threads())
            ref = np.asarray(ref).reshape(crop, crop, 6)
        got = out[0, :, :crop, :crop].float().cpu().numpy().transpose(1, 2, 0)
        err = got.astype(np.float64) - ref
        res[name] = {"ms": round(t, 3), "mpix_s": round(px / (t * 1e-3) / 1e6, 2),
                     "max_err_rel": float(np.abs(err).max() / np.abs(ref).max()),
                     "rms_err_rel": float(np.sqrt((err ** 2).mean()) / np.abs(ref).max())}
        if dt == torch.bfloat16:
            # the same BF16 image and bank through the tensor-core render
            ws = torch.empty(sd.api.render_tc_workspace(lay), dtype=torch.uint8, device=dev)
            t = _timed(lambda: sd.dp_render_tc(aif, depth, bank, lay, out=out, workspace=ws),
                       stream, reps=3)
            if int(ws[:4].view(torch.int32).item()) != 0:
                raise RuntimeError("tensor-core render: a completion wait gave up")
            got = out[0, :, :crop, :crop].float().cpu().numpy().transpose(1, 2, 0)
            err = got.astype(np.float64) - ref
            res["bf16_tc"] = {"ms": round(t, 3), "mpix_s": round(px / (t * 1e-3) / 1e6, 2),
                              "max_err_rel": float(np.abs(err).max() / np.abs(ref).max()),
                              "rms_err_rel": float(np.sqrt((err ** 2).mean()) / np.abs(ref).max())}
            del ws
        del out, bank
    res["bf16_speedup_vs_f32"] = round(res["f32"]["ms"] / res["bf16"]["ms"], 3)
    res["bf16_tc_speedup_vs_f32"] = round(res["f32"]["ms"] / res["bf16_tc"]["ms"], 3)
    res["bf16_bound"] = "max err <= 8 * 2^-9 of max|ref|"
    lens.free()
    return res


def pipeline_compare(sd, dev, reps=5):
    """Differentiation workload: trace the 32x32x3 bank at 128x128 pupil
    samples, render a batch of 8 RGB 512x512 images, render backward to the
    image and the bank, adjoint trace of the bank gradient.  Plain FP32 (one
    trace block per request, FP32 bank and images, eager launches) against
    the batched 16-bit pipelines, BF16 and FP16 (persistent batched trace
    writing a 16-bit bank, 16-bit images rendered on the tensor cores, FP32
    gradients: the image's on CUDA cores, the bank's on the tensor cores from
    weighted output gradients rounded to the 16-bit type; the whole step
    replayed from one CUDA graph).  Reported: each pipeline's time and
    stages, each bank's L1 error against the FP64 oracle, each 16-bit
    render's difference from the FP32 render."""
    import torch
    import oracle as O
    c = W.config_differentiation()
    H, Wd = c["image_hw"]
    B = c["batch"]
    reqs = W.bank_grid(c["field_h_mm"], c["depths_mm"], c["lambdas_nm"], c["n_grid"], c["ks"])
    n_req = len(reqs)
    lens = sd.Lens(c["lens"], c["focus_mm"])
    sensor = sd.DPSensor(c["pitch_mm"])
    req_dev, total, off = sd.make_requests(reqs, device=dev)
    aif_np = W.aif_pink(B, 3, H, Wd, seed=6).astype(np.float32)
    depth = torch.tensor(W.depth_perlin(B, H, Wd, seed=7).astype(np.float32), device=dev)
    gout = torch.randn((B, 6, H, Wd), device=dev, generator=torch.Generator(dev).manual_seed(1))
    fh, dm = c["field_h_mm"], c["depths_mm"] / 1000.0
    stream = torch.cuda.current_stream()
    ks = c["ks"]
    L = sd.lib()

    def make(dt):
        lay = sd.BankLayout(fh, dm, 3, ks, c["pitch_mm"], dtype=dt)
        aif = torch.tensor(aif_np, device=dev).to(dt)
        out = torch.empty((B, 6, H, Wd), dtype=dt, device=dev)
        gaif = torch.empty((B, 3, H, Wd), device=dev)
        gbank = torch.empty(total, device=dev)
        ws = torch.empty(sd.api.render_backward_workspace(lay, B, 3, H, Wd), dtype=torch.uint8,
                         device=dev)
        greq = torch.empty((n_req, 32, 8), device=dev)
        return lay, aif, out, gaif, gbank, ws, greq

    def render_bwd(lay, aif, bank, gaif, gbank, ws):
        lc = lay.c()
        sd._lib.check(L.sd_dp_render_backward(
            sd.api._ptr(gout), sd.api._ptr(aif), sd.api._ptr(depth), sd.api._ptr(bank),
            sd.api.ctypes.byref(lc), B, 3, H, Wd, sd.api._DT[aif.dtype], sd.api._ptr(gaif),
            sd.api._ptr(gbank) if gbank is not None else None, sd.api._ptr(ws), ws.numel(),
            sd.api._stream()), "sd_dp_render_backward")

    # plain FP32
    lay32, aif32, out32, gaif32, gbank32, ws32, greq32 = make(torch.float32)
    bank32 = torch.empty(total, device=dev)
    st32 = torch.zeros((n_req, 8), dtype=torch.int64, device=dev)

    # every pipeline's trace records the landing mask its adjoint reads
    mask32 = sd.land_mask(n_req, c["n_grid"], device=dev)

    def trace32():
        sd.dp_psf_trace(lens, sensor, req_dev, n_req, total, max_ks=ks, max_n=c["n_grid"],
                        norm=sd.SD_NORM_JOINT, out=bank32, stats=st32, mask=mask32)

    def adj(gb, greq, mask):
        sd.dp_psf_trace_backward(lens, sensor, req_dev, n_req, gb, max_ks=ks, max_n=c["n_grid"],
                                 grad_req=greq, mask=mask)

    def plain():
        trace32()
        sd.dp_render(aif32, depth, bank32, lay32, out=out32)
        render_bwd(lay32, aif32, bank32, gaif32, gbank32, ws32)
        adj(gbank32, greq32, mask32)

    t_plain = _timed(plain, stream, reps)
    stages = {"f32": {
        "trace": _timed(trace32, stream, reps),
        "render": _timed(lambda: sd.dp_render(aif32, depth, bank32, lay32, out=out32), stream,
                         reps),
        "render_bwd": _timed(lambda: render_bwd(lay32, aif32, bank32, gaif32, gbank32, ws32),
                             stream, reps),
        "trace_adjoint": _timed(lambda: adj(gbank32, greq32, mask32), stream, reps)}}
    torch.cuda.synchronize()
    r32 = out32.float()
    banks = {"f32": bank32.cpu().numpy()}
    res = {"requests": n_req, "rays": int(st32[:, 0].sum().item()), "images": [B, 3, H, Wd],
           "plain_f32_ms": round(t_plain, 3)}
    tune_cache = os.path.join(ROOT, "paper_2503_11213_gb300", "_build", "tune_cache.txt")
    for name, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        lay16, aif16, out16, gaif16, gbank16, ws16, greq16 = make(dt)
        mask16 = sd.land_mask(n_req, c["n_grid"], device=dev)
        bt = sd.BatchedTrace(lens, sensor, req_dev, n_req, total, max_ks=ks, max_n=c["n_grid"],
                             norm=sd.SD_NORM_JOINT, dtype=dt, mask=mask16)
        bt.tune(tune_cache)
        ws_tc = torch.empty(sd.api.render_tc_workspace(lay16), dtype=torch.uint8, device=dev)
        ws_bg = torch.empty(sd.api.bank_grad_tc_workspace(lay16, B, 3, H, Wd),
                            dtype=torch.uint8, device=dev)

        def render_bwd_tc():
            # image gradient on CUDA cores, bank gradient on the tensor cores
            render_bwd(lay16, aif16, bt.out, gaif16, None, ws16)
            sd.dp_render_bank_grad_tc(gout, aif16, depth, lay16, out=gbank16, workspace=ws_bg)

        def batched():
            bt.run()
            sd.dp_render_tc(aif16, depth, bt.out, lay16, out=out16, workspace=ws_tc)
            render_bwd_tc()
            adj(gbank16, greq16, mask16)

        s2 = torch.cuda.Stream()
        s2.wait_stream(stream)
        with torch.cuda.stream(s2):
            batched()
        stream.wait_stream(s2)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            batched()
        t_graph = _timed(g.replay, stream, reps)
        torch.cuda.synchronize()
        sd.sync_status(ws_tc[:4].view(torch.int32))
        sd.sync_status(ws_bg[:4].view(torch.int32))
        stages[name] = {
            "trace": _timed(lambda: bt.run(), stream, reps),
            "render": _timed(lambda: sd.dp_render_tc(aif16, depth, bt.out, lay16, out=out16,
                                                     workspace=ws_tc), stream, reps),
            "render_bwd": _timed(render_bwd_tc, stream, reps),
            "trace_adjoint": _timed(lambda: adj(gbank16, greq16, mask16), stream, reps)}
        torch.cuda.synchronize()
        res[f"batched_{name}_graph_ms"] = round(t_graph, 3)
        res[f"speedup_{name}"] = round(t_plain / t_graph, 3)
        res[f"render_max_rel_diff_{name}_vs_f32"] = float(
            (out16.float() - r32).abs().max().item() / r32.abs().max().item())
        banks[name] = bt.out.float().cpu().numpy()
        del g, bt, ws_tc, ws_bg, ws16, out16
    res["stages_ms"] = {k: {n: round(v, 3) for n, v in d.items()} for k, d in stages.items()}
    # bank error of every pipeline against the FP64 oracle on 24 evenly
    # spaced requests
    idx = np.linspace(0, n_req - 1, 24).astype(int)
    S = dict(ps=c["pitch_mm"], h=W.DP_H * c["pitch_mm"], f=W.DP_F * c["pitch_mm"],
             w=W.DP_W * c["pitch_mm"], r=W.DP_R * c["pitch_mm"])
    ref, _ = O.psf_bank(c["lens"], c["focus_mm"], reqs[idx], S, n_threads=cpu_threads())

    def l1(b):
        e = [np.abs(b[off[i]:off[i] + 2 * ks * ks] - r.ravel()).sum() / np.abs(r).sum()
             for i, r in zip(idx, ref)]
        return {"mean": float(np.mean(e)), "max": float(np.max(e))}

    res["bank_l1_vs_oracle"] = {k: l1(v) for k, v in banks.items()}
    res["bank_l1_vs_oracle"]["sample"] = "24 evenly spaced requests, FP64 oracle"
    lens.free()
    return res


PAPER_TRACE_S = 801.544   # DP PSF map of 512 x 768 pixels by ray tracing (Table S3)
PAPER_RENDER_S = 0.2      # DP image from a PSF map ("fixed cost", supplement)
PAPER_MLP_S = 0.395       # DP PSF map of 512 x 768 pixels by the MLP (supplement table)
MLP_FIT_ITERS = 30000     # Adam steps of the network fit in the paper-workload leg
MLP_FIT_POOL = 1 << 20    # traced points the fit draws its minibatches from


def quadrant_compare(sd, dev, reps=5):
    """The bench render (1024x1024 RGB, 65x65 kernels, doublet-pair lens)
    through a first-quadrant 2-D bank (16 x 16 field points up to the
    sensor's half width, 32 depths, 3 wavelengths; other quadrants by the
    PSF's flip symmetry) against the radial bank of the main step: trace
    and render times, and how far apart the two renders are."""
    import torch
    cfg = W.config_full_forward()
    H, Wd = cfg["sensor_hw"]
    ps = cfg["pitch_mm"]
    fq = np.linspace(0.0, 0.5 * Wd * ps, 16)
    lens = sd.Lens(cfg["lens"], cfg["focus_mm"])
    sensor = sd.DPSensor(ps)
    stream = torch.cuda.current_stream()
    aif = torch.tensor(W.aif_pink(1, 3, H, Wd, seed=1).astype(np.float32), device=dev)
    depth = torch.tensor(W.depth_perlin(1, H, Wd, seed=2).astype(np.float32), device=dev)
    dm = cfg["depths_mm"] / 1000.0
    res = {"field_points": [16, 16], "depths": len(dm), "lambdas": 3, "ks": cfg["ks"],
           "pupil_grid": [cfg["n_grid"]] * 2, "image": [1, 3, H, Wd]}
    outs = {}
    for name, fh, mode, reqs in (
            ("radial", cfg["field_h_mm"], sd.SD_FIELD_RADIAL,
             W.bank_grid(cfg["field_h_mm"], cfg["depths_mm"], cfg["lambdas_nm"], cfg["n_grid"],
                         cfg["ks"])),
            ("quadrant", fq, sd.SD_FIELD_QUADRANT,
             W.bank_grid_quadrant(fq, cfg["depths_mm"], cfg["lambdas_nm"], cfg["n_grid"],
                                  cfg["ks"]))):
        req_dev, total, _ = sd.make_requests(reqs, device=dev)
        bank = torch.empty(total, device=dev)
        st = torch.zeros((len(reqs), 8), dtype=torch.int64, device=dev)
        t_trace = _timed(lambda: sd.dp_psf_trace(lens, sensor, req_dev, len(reqs), total,
                                                 max_ks=cfg["ks"], max_n=cfg["n_grid"],
                                                 norm=sd.SD_NORM_JOINT, out=bank, stats=st),
                         stream, reps=3)
        lay = sd.BankLayout(fh, dm, 3, cfg["ks"], ps, field_mode=mode)
        out = torch.empty((1, 6, H, Wd), device=dev)
        t_render = _timed(lambda: sd.dp_render(aif, depth, bank, lay, out=out), stream, reps)
        outs[name] = out
        res[name] = {"psfs": len(reqs), "rays": int(st[:, 0].sum().item()),
                     "trace_ms": round(t_trace, 3), "render_ms": round(t_render, 3)}
        del bank
    ref = outs["radial"]
    res["max_rel_diff_quadrant_vs_radial"] = float(
        ((outs["quadrant"] - ref).abs().max() / ref.abs().max()).item())
    lens.free()
    return res


def paper_workload(sd, dev, reps=5):
    """The paper's own timed path (Sec. 5.1 implementation details, Table S3):
    RF50 (Table S1) at F/4, 550 nm, focus 1 m, a DP PSF for every pixel of a
    512 x 768 depth map over 0.5-20 m (64 x 64 pupil grid = 4096 samples,
    21 x 21 patches), then the DP render of a 512 x 768 RGB image from that
    map.  The paper's times (its i7-12700K + RTX 3090) are context."""
    import torch
    c = W.config_paper_rf50()
    H, Wd = c["sensor_hw"]
    tab = sd.f_number_table(c["lens"], c["f_number"], c["lambda_nm"], c["focus_mm"])
    lens = sd.Lens(tab, c["focus_mm"])
    sensor = sd.DPSensor(c["pitch_mm"])
    depth = torch.tensor(W.depth_perlin(1, H, Wd, seed=8, d_near_m=c["d_near_m"],
                                        d_far_m=c["d_far_m"])[0].astype(np.float32), device=dev)
    aif = torch.tensor(W.aif_pink(1, 3, H, Wd, seed=9).astype(np.float32), device=dev)
    stream = torch.cuda.current_stream()
    ks, n = c["ks"], c["n_grid"]
    res = {"lens": "RF50 (Table S1) at F/4", "lambda_nm": c["lambda_nm"],
           "map": [H, Wd, 2, ks, ks], "pupil_grid": [n, n], "depth_m": [0.5, 20.0],
           "paper_trace_s": PAPER_TRACE_S, "paper_render_s": PAPER_RENDER_S,
           "paper_hardware": "i7-12700K + RTX 3090 (context, not the target)"}
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        pmap = torch.empty((H, Wd, 2, ks, ks), dtype=dt, device=dev)
        stats = torch.zeros((H * Wd, 8), dtype=torch.int64, device=dev)
        img = aif if dt == torch.float32 else aif.to(dt)
        out = torch.empty((1, 6, H, Wd), dtype=dt, device=dev)
        t_tr = _timed(lambda: sd.dp_psf_map(lens, sensor, depth, c["lambda_nm"], n, ks,
                                            out=pmap, stats=stats), stream, reps)
        # the bulk-copy form (with a status word) and the per-thread-load form
        st_r = torch.empty(1, dtype=torch.int32, device=dev)
        t_rd = _timed(lambda: sd.dp_render_map(img, pmap, out=out, status=st_r), stream, reps)
        sd.sync_status(st_r)
        t_rd_loads = _timed(lambda: sd.dp_render_map(img, pmap, out=out, status=False), stream,
                            reps)
        rays = int(stats[:, 0].sum().item())
        map_bytes = pmap.numel() * pmap.element_size()
        io_bytes = img.numel() * img.element_size() + out.numel() * out.element_size()
        res[name] = {"trace_ms": round(t_tr, 3), "render_ms": round(t_rd, 4),
                     "psfs_per_s": round(H * Wd / (t_tr * 1e-3), 1),
                     "rays": rays, "grays_s": round(rays / (t_tr * 1e-3) / 1e9, 3),
                     "render_gbs": round((map_bytes + io_bytes) / (t_rd * 1e-3) / 1e9, 1),
                     "render_ms_per_thread_loads": round(t_rd_loads, 4),
                     "trace_speedup_vs_paper": round(PAPER_TRACE_S / (t_tr * 1e-3), 1),
                     "render_speedup_vs_paper": round(PAPER_RENDER_S / (t_rd * 1e-3), 1)}
        if dt == torch.float32:
            traced_map = pmap   # the reference of the fitted network below
        del pmap, out
    peaks = load_peaks()
    if peaks.get("hbm_gbs"):
        res["render_hbm_frac_f32"] = round(res["f32"]["render_gbs"] / peaks["hbm_gbs"], 3)
        res["render_hbm_frac_bf16"] = round(res["bf16"]["render_gbs"] / peaks["hbm_gbs"], 3)
    # the paper's render-time PSF source: the network of Sec. 3.2 (5 x 512,
    # 2 ks^2 outputs) fitted to PSFs traced at random points of the region
    # (max-normalised targets, Eq. 4 loss; seeded), its tensor-core map of
    # every pixel, then the same render from that map
    from paper_2503_11213_gb300 import psf_net as PN
    ws, bs, info = PN.fit(lens, sensor, (H, Wd), c["pitch_mm"], c["d_near_m"], c["d_far_m"],
                          c["lambda_nm"], n, ks, iters=MLP_FIT_ITERS, batch=1024,
                          pool=MLP_FIT_POOL, seed=0, device=dev)
    net = sd.PsfMLP(ws, bs, ks)
    shapes = sd.MLP_SHAPES(ks)
    flops = 2.0 * H * Wd * sum(a * b for a, b in shapes)
    mlp = {"network": "3 -> 5 x 512 (ReLU) -> 2 ks^2, fitted to traced PSFs",
           "fit": {"iters": info["iters"], "batch": info["batch"], "pool_points": info["pool"],
                   "pool_trace_s": round(info["trace_s"], 3), "train_s": round(info["train_s"], 2),
                   "first_loss": info["first_loss"], "final_loss": info["final_loss"],
                   "seed": info["seed"]},
           "paper_mlp_s": PAPER_MLP_S, "flops_per_map": flops}
    st = torch.empty(1, dtype=torch.int32, device=dev)
    for name, dt in (("f32_map", torch.float32), ("bf16_map", torch.bfloat16)):
        pmap = torch.empty((H, Wd, 2, ks, ks), dtype=dt, device=dev)
        img = aif if dt == torch.float32 else aif.to(dt)
        out = torch.empty((1, 6, H, Wd), dtype=dt, device=dev)
        t_m = _timed(lambda: sd.mlp_psf_map(net, depth, c["d_near_m"], c["d_far_m"], out=pmap,
                                            status=st), stream, reps)
        sd.sync_status(st)

        def both():
            sd.mlp_psf_map(net, depth, c["d_near_m"], c["d_far_m"], out=pmap, status=st)
            sd.dp_render_map(img, pmap, out=out)
        t_b = _timed(both, stream, reps)
        tf = flops / (t_m * 1e-3) / 1e12
        mlp[name] = {"mlp_map_ms": round(t_m, 3), "mlp_map_plus_render_ms": round(t_b, 3),
                     "tflops": round(tf, 1),
                     "frac_of_bf16_peak": round(tf / peaks["bf16_tflops"], 3)
                     if peaks.get("bf16_tflops") else None,
                     "speedup_vs_paper_mlp": round(PAPER_MLP_S / (t_m * 1e-3), 1)}
        if dt == torch.float32:
            # accuracy of the predicted map against the traced map of the same
            # depth map (per element of the sum-normalised PSFs), split into
            # the fit (the FP32 network) and the kernel's BF16 activations
            yy, xx = torch.meshgrid(torch.arange(H, device=dev), torch.arange(Wd, device=dev),
                                    indexing="ij")
            pin = torch.stack([(xx - 0.5 * (Wd - 1)) / (0.5 * Wd),
                               (yy - 0.5 * (H - 1)) / (0.5 * H),
                               2 * (depth - c["d_near_m"]) / (c["d_far_m"] - c["d_near_m"]) - 1],
                              -1).reshape(-1, 3).float()
            prm = [torch.tensor(a, device=dev) for pair in zip(ws, bs) for a in pair]
            with torch.no_grad():
                f32net = torch.cat([PN.sum_normalised(PN.forward(prm, pin[i:i + 65536]))
                                    for i in range(0, pin.shape[0], 65536)]).view(pmap.shape)
            # the traced map itself carries the sampling noise of 4096 rays;
            # a 256 x 256-ray trace of the same pixels shows what the fit
            # reaches against a nearly noise-free reference
            fine, _ = sd.dp_psf_map(lens, sensor, depth, c["lambda_nm"], 256, ks)
            mlp["accuracy_vs_traced_map"] = {
                "kernel_map": PN.map_errors(pmap, traced_map),
                "fp32_network": PN.map_errors(f32net, traced_map),
                "kernel_vs_fp32_network": PN.map_errors(pmap, f32net),
                "kernel_map_vs_65536_ray_map": PN.map_errors(pmap, fine),
                "traced_map_vs_65536_ray_map": PN.map_errors(traced_map, fine),
                "definition": "per element of the sum-normalised 2 x 21 x 21 PSFs of all "
                              "512 x 768 pixels: l1 = mean |err|, l2 = mean err^2",
                "paper_table_s3": {"l1": 6.887e-5, "l2": 6.830e-8,
                                   "note": "50 depths and positions, RTX 3090; context"}}
            del f32net, fine
        del pmap, out
    del traced_map
    res["mlp"] = mlp
    lens.free()
    return res


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(cfg, reqs, aif_np, depth_np, budget_s):
    """The FP64 oracle, as it stands, on a bounded sample of each phase of
    the same step, each phase's time scaled linearly to the full step:
    the trace (every k-th bank request, threads over requests), the render
    (a set of pixels, threads over pixels), the render backward (an image
    crop, the oracle's single-threaded adjoint) and the adjoint trace
    (evenly spaced live requests, threads over requests, forward-mode dual
    numbers for the 22 lens parameters of the differentiation study: its
    cost does not depend on the gradient's values)."""
    import oracle as O
    cores = cpu_threads()
    ps = cfg["pitch_mm"]
    S = dict(ps=ps, h=W.DP_H * ps, f=W.DP_F * ps, w=W.DP_W * ps, r=W.DP_R * ps)
    n_req = len(reqs)
    lens, focus = cfg["lens"], cfg["focus_mm"]
    # trace: calibrate on one request, then fill about 0.3 of the budget
    t0 = time.perf_counter()
    O.psf_bank(lens, focus, reqs[:1], S, n_threads=1)
    per_req = time.perf_counter() - t0
    n_s = int(max(cores, min(n_req, round(0.3 * budget_s * cores / max(per_req, 1e-6)))))
    n_s = max(cores, (n_s // cores) * cores)
    idx = np.linspace(0, n_req - 1, n_s).astype(int)
    t0 = time.perf_counter()
    _, st = O.psf_bank(lens, focus, reqs[idx], S, n_threads=cores)
    t_trace = (time.perf_counter() - t0) * n_req / n_s
    rays = int(st[:, 0].sum()) * n_req / n_s
    # render: a set of pixels
    cfgd = cfg["depths_mm"] / 1000.0
    rng = np.random.default_rng(0)
    nf, nz = len(cfg["field_h_mm"]), len(cfgd)
    bank = np.full((nf, nz, 3, 2, cfg["ks"], cfg["ks"]), 1.0 / (2 * cfg["ks"] ** 2))
    H, Wd = aif_np.shape[2:]
    npx = 64 * cores
    pix = np.stack([np.zeros(npx, int), rng.integers(0, H, npx), rng.integers(0, Wd, npx)], 1)
    t0 = time.perf_counter()
    O.render_bank_pixels(aif_np, depth_np, bank, cfg["field_h_mm"], cfgd, ps, pix,
                         n_threads=cores)
    t_render = (time.perf_counter() - t0) * (H * Wd) / npx
    # render backward: an image crop, side calibrated on 8 x 8 pixels to
    # about 0.2 of the budget
    def bwd_crop(side):
        y0, x0 = (H - side) // 2, (Wd - side) // 2
        a = aif_np[:, :, y0:y0 + side, x0:x0 + side]
        g = rng.standard_normal((1, 6, side, side))
        d = depth_np[:, y0:y0 + side, x0:x0 + side]
        t0 = time.perf_counter()
        O.render_bank_bwd(g, a, d, bank, cfg["field_h_mm"], cfgd, ps)
        return time.perf_counter() - t0
    t8 = bwd_crop(8)
    side = int(np.clip(8 * np.sqrt(0.2 * budget_s / max(t8, 1e-6)), 8, min(H, Wd)))
    t_bwd = bwd_crop(side) * (H * Wd) / (side * side)
    # adjoint: the requests whose slice some pixel uses (the others have a
    # zero gradient patch), sampled evenly, traced at 64 x 64 pupil samples
    # and scaled by the rays the step's requests launch
    sel = O.render_select(depth_np[0], cfg["field_h_mm"], cfgd, ps)
    f, z0, t = sel[..., 0].astype(int), sel[..., 1].astype(int), sel[..., 3]
    used = np.zeros(nf * nz, bool)
    used[(f * nz + z0)[t < 1]] = True
    up = (t > 0) & (z0 + 1 < nz)
    used[(f * nz + z0 + 1)[up]] = True
    nl = n_req // (nf * nz)
    live = np.flatnonzero(np.repeat(used, nl))
    pids = [O.param_id(s_, "c") for s_ in range(1, 7)] + [O.param_id(1, "k"), O.param_id(6, "k")]
    pids += [O.param_id(s_, a_) for s_ in (1, 6) for a_ in ("a4", "a6", "a8", "a10")]
    pids += [O.param_id(s_, "t") for s_ in range(1, 7)]
    small = reqs.copy()
    small["n_grid"] = 64
    G1 = [rng.standard_normal((2, cfg["ks"], cfg["ks"]))]
    t0 = time.perf_counter()
    O.trace_grad(lens, focus, small[live[:1]], S, G1, pids, n_threads=1)
    per_adj = time.perf_counter() - t0
    n_a = int(max(cores, min(len(live), round(0.2 * budget_s * cores / max(per_adj, 1e-6)))))
    n_a = max(1, min(len(live), (n_a // cores) * cores or cores))
    aidx = live[np.linspace(0, len(live) - 1, n_a).astype(int)]
    G = [rng.standard_normal((2, cfg["ks"], cfg["ks"])) for _ in range(n_a)]
    _, st_small = O.psf_bank(lens, focus, small[aidx[:1]], S, n_threads=1)
    t0 = time.perf_counter()
    O.trace_grad(lens, focus, small[aidx], S, G, pids, n_threads=cores)
    ray_scale = (int(st[:, 0].sum()) / n_s) / max(1, int(st_small[0, 0]))
    t_adj = (time.perf_counter() - t0) * len(live) / n_a * ray_scale
    step_s = t_trace + t_render + t_bwd + t_adj
    return {"value": round(rays / step_s / 1e9, 6), "unit": "G rays/s", "cores": cores,
            "kind": "oracle",
            "sample": f"trace: {n_s} of {n_req} bank requests (evenly spaced); render: {npx} "
                      f"of {H * Wd} pixels; render backward: a {side}x{side} crop (the "
                      f"oracle's adjoint is single-threaded); adjoint: {n_a} of the "
                      f"{len(live)} requests with a non-zero gradient patch at 64x64 pupil "
                      f"samples, scaled by launched rays (x{ray_scale:.1f}); FP64 C++ oracle "
                      f"on {cores} threads, each phase scaled linearly to the full step",
            "step_s_extrapolated": round(step_s, 3),
            "trace_s": round(t_trace, 3), "render_s": round(t_render, 3),
            "render_bwd_s": round(t_bwd, 3), "adjoint_s": round(t_adj, 3)}


def run_reference(args, world, rank):
    """The oracle as the reference arm: each step is a bounded sample of the
    workload timed on the host cores (rank 0 only)."""
    if rank != 0:
        return None
    cfg, reqs, aif_np, depth_np = build_inputs(None)
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(cfg, reqs, aif_np, depth_np, per_step)
    vals = []
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(cfg, reqs, aif_np, depth_np, per_step)
        vals.append(last["value"])
    value = statistics.mean(vals)
    step_ms = last["step_s_extrapolated"] * 1e3
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "G rays/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(step_ms, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD}, "cpu_baseline": last,
            "e2e": {"value": value, "unit": "G rays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the differentiation-pipeline and precision legs")
    ap.add_argument("--requests", type=int, default=0,
                    help="profiling only: trace every k-th bank request")
    ap.add_argument("--image", type=int, default=0, help="profiling only: render size")
    args = ap.parse_args()
    world, rank, local, dist = setup_dist(args)
    if args.impl == "reference":
        line = run_reference(args, world, rank)
    else:
        line = run_ours(args, world, rank, local, dist)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
