"""torch.autograd.Function wrappers of the render and of the trace.

Both backward passes call the hand-written adjoint kernels of the CUDA
library (render backward; adjoint trace, which recomputes the rays instead of
storing them between the passes).  Only marshalling happens here.
"""
from __future__ import annotations

import torch

from . import _lib as L
from .api import BankLayout, DPSensor, Lens, dp_psf_trace, dp_psf_trace_backward, dp_render, \
    dp_render_backward, land_mask


class DPRenderFunction(torch.autograd.Function):
    """(aif, bank) -> DP image (N, 2C, H, W) through the per-pixel DP PSF
    render of the supplement's local DP PSF convolution; the depth map selects
    the bank slices and is not differentiated (the selection is piecewise
    constant in depth apart from the linear interpolation weight)."""

    @staticmethod
    def forward(ctx, aif, bank, depth_m, layout: BankLayout):
        out = dp_render(aif, depth_m, bank, layout)
        ctx.save_for_backward(aif, bank, depth_m)
        ctx.layout = layout
        return out

    @staticmethod
    def backward(ctx, grad_out):
        aif, bank, depth_m = ctx.saved_tensors
        need_aif, need_bank = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_aif or need_bank):
            return None, None, None, None
        g = grad_out.to(torch.float32).contiguous()
        ga, gb = dp_render_backward(g, aif, depth_m, bank, ctx.layout, need_aif=need_aif,
                                    need_bank=need_bank)
        return ga, gb, None, None


def dp_render_autograd(aif, bank, depth_m, layout: BankLayout):
    """dp_render with gradients for aif and bank (FP32) through the render
    adjoint of the CUDA library."""
    return DPRenderFunction.apply(aif, bank, depth_m, layout)


class DPTraceFunction(torch.autograd.Function):
    """Lens parameters -> PSF bank (bilinear splat, Eq. 3 with the unit ray
    energy spread over the four nearest pixel centres), differentiable with
    respect to the selected parameters.

    theta: 1-D tensor of parameter values, one per id in ``pids`` (id =
    surface * 8 + j with j = curvature, conic, a4..a12, thickness after the
    surface; the last surface's thickness is the sensor distance).  The
    forward writes theta into the lens (host side) before tracing.  Ray
    generation (object point, entrance pupil, patch centre) follows the lens
    as set, and its dependence on theta is not differentiated; the L/R and
    base-pixel decisions are those of the forward pass.
    """

    @staticmethod
    def forward(ctx, theta, lens: Lens, pids, sensor: DPSensor, req_dev, n_req, total,
                max_ks, max_n, norm):
        if norm not in (L.SD_NORM_NONE, L.SD_NORM_PER_RAY):
            raise ValueError("the adjoint trace differentiates SD_NORM_NONE or SD_NORM_PER_RAY")
        vals = theta.detach().to("cpu", torch.float64).tolist()
        for pid, v in zip(pids, vals):
            lens.set_param(int(pid), float(v))
        # the rays that land near their patch, so that the backward traces
        # only those again (the lens stays as set here until then)
        mask = land_mask(n_req, max_n, device=req_dev.device)
        out, _ = dp_psf_trace(lens, sensor, req_dev, n_req, total, max_ks=max_ks, max_n=max_n,
                              mode=L.SD_BIN_BILINEAR, norm=norm, mask=mask)
        ctx.mask = mask
        ctx.lens, ctx.pids, ctx.sensor = lens, list(pids), sensor
        ctx.req_dev, ctx.n_req, ctx.max_ks, ctx.max_n, ctx.norm = req_dev, n_req, max_ks, max_n, norm
        ctx.theta_meta = (theta.dtype, theta.device)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.to(torch.float32).contiguous()
        _, grad_lens = dp_psf_trace_backward(ctx.lens, ctx.sensor, ctx.req_dev, ctx.n_req, g,
                                             max_ks=ctx.max_ks, max_n=ctx.max_n, norm=ctx.norm,
                                             mask=ctx.mask)
        flat = grad_lens[0].reshape(-1)
        idx = torch.tensor(ctx.pids, dtype=torch.long, device=flat.device)
        dtype, device = ctx.theta_meta
        gtheta = flat.index_select(0, idx).to(device=device, dtype=dtype)
        return (gtheta,) + (None,) * 9


def dp_psf_trace_autograd(theta, lens: Lens, pids, sensor: DPSensor, req_dev, n_req, total,
                          max_ks, max_n=512, norm=L.SD_NORM_PER_RAY):
    """Bilinear PSFs of the requests as a function of the lens parameters
    theta (the parameter ids pids of lens), with gradients through the
    adjoint trace; norm is per-ray or none (a joint normalisation has no
    useful gradient)."""
    return DPTraceFunction.apply(theta, lens, pids, sensor, req_dev, n_req, total, max_ks,
                                 max_n, norm)
