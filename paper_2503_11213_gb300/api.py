"""PyTorch-facing API of the DP simulator hot path.

Every function marshals tensors into the C ABI of include/sdirt.h and runs on
the current CUDA stream; all arithmetic happens in the CUDA library.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

_DT = {torch.float32: L.SD_F32, torch.bfloat16: L.SD_BF16, torch.float16: L.SD_F16}


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError("expected contiguous CUDA tensors")


@dataclass
class DPSensor:
    """DP pixel structure (Sec. 3.1); defaults are Eq. (S1) multiples of ps."""
    pitch_mm: float
    h: float = 0.78
    f: float = 1.44
    w: float = 0.30
    r: float = 0.50

    def c(self):
        ps = self.pitch_mm
        return L.SdSensor(ps, self.h * ps, self.f * ps, self.w * ps, self.r * ps)


class Lens:
    """A lens prescription uploaded to the device lens table.

    table: (n, 12) float64 rows (type, radius, thickness, nd, vd,
    semi-diameter, conic, a4..a12), as produced by ``workloads``.
    """

    def __init__(self, table, focus_mm: float = 0.0):
        lib = L.lib()
        tab = np.asarray(table, dtype=np.float64)
        n = tab.shape[0]
        arr = (L.SdSurface * n)()
        for i, r in enumerate(tab):
            s = arr[i]
            s.type = int(r[0])
            s.radius, s.thickness, s.nd, s.vd, s.semi_diameter, s.conic = map(float, r[1:7])
            for j in range(5):
                s.asph[j] = float(r[7 + j])
        h = ctypes.c_void_p()
        L.check(lib.sd_lens_load(arr, n, float(focus_mm), ctypes.byref(h)), "sd_lens_load")
        self._h = h
        self.n_surfaces = n

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("lens already freed")
        return self._h

    def paraxial(self, lambda_nm=587.5618, depth_mm=1000.0):
        out = L.SdParaxial()
        L.check(L.lib().sd_lens_paraxial(self.handle, float(lambda_nm), float(depth_mm),
                                         ctypes.byref(out)), "sd_lens_paraxial")
        return {k: getattr(out, k) for k, _ in L.SdParaxial._fields_}

    def set_param(self, param_id: int, value: float):
        L.check(L.lib().sd_lens_set_param(self.handle, int(param_id), float(value)),
                "sd_lens_set_param")

    def free(self):
        if self._h is not None:
            L.lib().sd_lens_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def make_requests(reqs, ks_offsets=True, device="cuda"):
    """Structured numpy requests (fields h_mm, depth_mm, lambda_nm, n_grid, ks
    and optionally lens) -> (device uint8 tensor of sd_psf_request, total
    output elements, per-request offsets)."""
    n = len(reqs)
    rec = np.zeros(n, dtype=L.REQUEST_DTYPE)
    for f in ("h_mm", "depth_mm", "lambda_nm", "n_grid", "ks"):
        rec[f] = reqs[f]
    for f in ("lens", "v_mm"):
        if f in reqs.dtype.names:
            rec[f] = reqs[f]
    sizes = 2 * rec["ks"].astype(np.int64) ** 2
    off = np.zeros(n, dtype=np.int64)
    off[1:] = np.cumsum(sizes)[:-1]
    rec["out_offset"] = off
    total = int(sizes.sum())
    dev = torch.from_numpy(rec.view(np.uint8).copy()).to(device)
    return dev, total, off


def check_status():
    """Bounds checks of the checked build (SDIRT_CHECKED=1): synchronises the
    device, then returns and clears (site, index, bound, count): the first
    failing check's site (translation unit * 100000 + source line; 0 if
    none), its index and bound, and the number of failed checks.  Raises
    SdError (SD_ERR_UNSUPPORTED) in the normal build."""
    site, index, bound = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
    count = ctypes.c_int64(0)
    L.check(L.lib().sd_check_status(ctypes.byref(site), ctypes.byref(index), ctypes.byref(bound),
                                    ctypes.byref(count)), "sd_check_status")
    return site.value, index.value, bound.value, count.value


def land_mask_bytes(n_req, max_n=512):
    """Bytes of a landing mask (sd_dp_psf_trace_mask_bytes)."""
    n = ctypes.c_size_t(0)
    L.check(L.lib().sd_dp_psf_trace_mask_bytes(n_req, max_n, ctypes.byref(n)),
            "sd_dp_psf_trace_mask_bytes")
    return n.value


def land_mask(n_req, max_n=512, device="cuda"):
    """An uninitialised landing mask for n_req requests (int32 words): pass
    it to dp_psf_trace to record which rays land near the patch, then to
    dp_psf_trace_backward of the same lenses, sensor and requests."""
    return torch.empty(max(1, land_mask_bytes(n_req, max_n) // 4), dtype=torch.int32,
                       device=device)


def _mask_ptr(mask):
    if mask is None:
        return None
    _need_cuda(mask)
    if mask.dtype != torch.int32:
        raise ValueError("the landing mask must be an int32 tensor (land_mask())")
    return mask.data_ptr()


def dp_psf_trace(lenses, sensor: DPSensor, req_dev, n_req, total, max_ks, max_n=512,
                 mode=L.SD_BIN_HARD, norm=L.SD_NORM_JOINT, dtype=torch.float32,
                 out=None, stats=None, newton_iters=0, mask=None):
    """Traces the requests (device array from make_requests) into a flat bank.
    mask (from land_mask(n_req, max_n)), if given, records for every ray
    whether it lands within a pixel of its request's patch."""
    lenses = lenses if isinstance(lenses, (list, tuple)) else [lenses]
    handles = (ctypes.c_void_p * len(lenses))(*[l.handle.value for l in lenses])
    if out is None:
        out = torch.empty(total, dtype=dtype, device=req_dev.device)
    if stats is None:
        stats = torch.zeros((n_req, L.SD_N_STATS), dtype=torch.int64, device=req_dev.device)
    _need_cuda(req_dev, out, stats)
    if mask is not None and mask.numel() * 4 < land_mask_bytes(n_req, max_n):
        raise ValueError("the landing mask is too small for these requests")
    opts = L.SdTraceOpts(mode, norm, _DT[out.dtype], newton_iters, max_ks, max_n,
                         _mask_ptr(mask))
    sen = sensor.c()
    L.check(L.lib().sd_dp_psf_trace(handles, len(lenses), ctypes.byref(sen), _ptr(req_dev),
                                    n_req, ctypes.byref(opts), _ptr(out), _ptr(stats),
                                    _stream()), "sd_dp_psf_trace")
    return out, stats


def dp_psf_trace_backward(lenses, sensor: DPSensor, req_dev, n_req, grad_out, max_ks,
                          max_n=512, norm=L.SD_NORM_PER_RAY, grad_req=None, newton_iters=0,
                          swept=None, mask=None):
    """Adjoint of the bilinear trace: per-request and per-lens gradients of
    <grad_out, PSF> with respect to the lens parameters, as
    (grad_req (n_req, 32, 8), grad_lens (n_lenses, 32, 8)).  swept, an
    optional (n_req, 2) int64 CUDA tensor, receives per request the rays with
    a non-zero splat gradient and the ray slots that ran the sweep (two per thread).  mask,
    a landing mask written by dp_psf_trace of the same lenses, sensor and
    requests (same max_n), restricts the retrace to the rays it marks."""
    lenses = lenses if isinstance(lenses, (list, tuple)) else [lenses]
    handles = (ctypes.c_void_p * len(lenses))(*[l.handle.value for l in lenses])
    dev = req_dev.device
    if grad_req is None:
        grad_req = torch.empty((n_req, L.SD_MAX_SURFACES, L.NPAR_SURF), device=dev)
    grad_lens = torch.empty((len(lenses), L.SD_MAX_SURFACES, L.NPAR_SURF), device=dev)
    _need_cuda(req_dev, grad_out, grad_req)
    if swept is not None:
        _need_cuda(swept)
        if swept.dtype != torch.int64 or swept.numel() < 2 * n_req:
            raise ValueError("swept must be an int64 tensor of n_req x 2")
    if mask is not None and mask.numel() * 4 < land_mask_bytes(n_req, max_n):
        raise ValueError("the landing mask is too small for these requests")
    opts = L.SdTraceOpts(L.SD_BIN_BILINEAR, norm, L.SD_F32, newton_iters, max_ks, max_n,
                         _mask_ptr(mask))
    sen = sensor.c()
    L.check(L.lib().sd_dp_psf_trace_backward(handles, len(lenses), ctypes.byref(sen),
                                             _ptr(req_dev), n_req, ctypes.byref(opts),
                                             _ptr(grad_out), _ptr(grad_req), _ptr(grad_lens),
                                             _ptr(swept) if swept is not None else None,
                                             _stream()), "sd_dp_psf_trace_backward")
    return grad_req, grad_lens


def dp_psf_map(lens: Lens, sensor: DPSensor, depth_m, lambda_nm, n_grid, ks,
               mode=L.SD_BIN_HARD, norm=L.SD_NORM_JOINT, dtype=torch.float32, out=None,
               stats=None, newton_iters=0):
    """Per-pixel DP PSF map of an (H, W) depth map (metres, float32, CUDA):
    (map (H, W, 2, ks, ks) in dtype, stats (H*W, 8))."""
    H, W = depth_m.shape
    dev = depth_m.device
    if out is None:
        out = torch.empty((H, W, 2, ks, ks), dtype=dtype, device=dev)
    if stats is None:
        stats = torch.zeros((H * W, L.SD_N_STATS), dtype=torch.int64, device=dev)
    _need_cuda(depth_m, out, stats)
    if depth_m.dtype != torch.float32:
        raise ValueError("depth must be float32 metres")
    opts = L.SdTraceOpts(mode, norm, _DT[out.dtype], newton_iters, ks, n_grid)
    sen = sensor.c()
    L.check(L.lib().sd_dp_psf_map(lens.handle, ctypes.byref(sen), _ptr(depth_m), H, W,
                                  float(lambda_nm), int(n_grid), int(ks), ctypes.byref(opts),
                                  _ptr(out), _ptr(stats), _stream()), "sd_dp_psf_map")
    return out, stats


def dp_render_map(aif, psf_map, out=None, status=None):
    """aif (N,C,H,W) f32/bf16/f16 and a PSF map (H,W,2,ks,ks) -> DP image
    (N,2C,H,W) in aif's dtype (one kernel pair per pixel for all channels).
    status: a device int32 word (one is made if None) that the call zeroes
    and sets to 1 if a bounded wait of the bulk-copy form gave up; read it
    with sync_status.  status=False takes the per-thread-load form."""
    N, C, H, W = aif.shape
    ks = psf_map.shape[-1]
    if tuple(psf_map.shape) != (H, W, 2, ks, ks):
        raise ValueError("psf_map must be (H, W, 2, ks, ks)")
    if out is None:
        out = torch.empty((N, 2 * C, H, W), dtype=aif.dtype, device=aif.device)
    if status is None:
        status = torch.empty(1, dtype=torch.int32, device=aif.device)
    _need_cuda(aif, psf_map, out, *([status] if status is not False else []))
    L.check(L.lib().sd_dp_render_map(_ptr(aif), _ptr(psf_map), N, C, H, W, ks, _DT[aif.dtype],
                                     _DT[psf_map.dtype], _ptr(out),
                                     None if status is False else _ptr(status), _stream()),
            "sd_dp_render_map")
    return out


def f_number_table(table, f_number, lambda_nm=587.5618, focus_mm=1000.0):
    """A copy of a lens table with the stop's semi-diameter scaled so that
    EFL / (2 r_EP) = f_number at lambda_nm (paraxial; the entrance-pupil
    radius is proportional to the stop radius)."""
    tab = np.array(table, dtype=np.float64, copy=True)
    lens = Lens(tab, focus_mm)
    try:
        px = lens.paraxial(lambda_nm, focus_mm)
    finally:
        lens.free()
    stop = int(np.nonzero(tab[:, 0] == L.SD_SURF_STOP)[0][0])
    tab[stop, 5] *= (px["efl"] / (2.0 * f_number)) / px["r_ep"]
    return tab


def batched_workspace_bytes(n_req, total):
    """Device workspace bytes of the batched trace of n_req requests writing
    total output elements (sd_dp_psf_trace_batched_workspace)."""
    n = ctypes.c_size_t(0)
    L.check(L.lib().sd_dp_psf_trace_batched_workspace(n_req, total, ctypes.byref(n)),
            "sd_dp_psf_trace_batched_workspace")
    return n.value


class BatchedTrace:
    """Uneven requests traced in one persistent launch (hard binning).

    Holds the output, statistics and workspace so that ``run()`` allocates
    nothing and can be captured in a CUDA graph."""

    def __init__(self, lenses, sensor: DPSensor, req_dev, n_req, total, max_ks, max_n=512,
                 norm=L.SD_NORM_JOINT, dtype=torch.float32, config=None, mask=None):
        self.lenses = lenses if isinstance(lenses, (list, tuple)) else [lenses]
        self.handles = (ctypes.c_void_p * len(self.lenses))(
            *[l.handle.value for l in self.lenses])
        dev = req_dev.device
        self.req_dev, self.n_req, self.total = req_dev, n_req, total
        self.out = torch.empty(total, dtype=dtype, device=dev)
        self.stats = torch.zeros((n_req, L.SD_N_STATS), dtype=torch.int64, device=dev)
        self.ws = torch.empty(batched_workspace_bytes(n_req, total), dtype=torch.uint8, device=dev)
        self.sen = sensor.c()
        # mask (from land_mask(n_req, max_n)), if given, receives every
        # ray's landing bit on each run, as dp_psf_trace writes it
        if mask is not None and mask.numel() * 4 < land_mask_bytes(n_req, max_n):
            raise ValueError("the landing mask is too small for these requests")
        self.mask = mask
        self.opts = L.SdTraceOpts(L.SD_BIN_HARD, norm, _DT[dtype], 0, max_ks, max_n,
                                  _mask_ptr(mask))
        self.config = L.SdBatchConfig(*(config or (0, 0, 0)), 0)

    def run(self):
        L.check(L.lib().sd_dp_psf_trace_batched(
            self.handles, len(self.lenses), ctypes.byref(self.sen), _ptr(self.req_dev),
            self.n_req, ctypes.byref(self.opts), ctypes.byref(self.config), _ptr(self.out),
            self.total, _ptr(self.stats), _ptr(self.ws), self.ws.numel(), _stream()),
            "sd_dp_psf_trace_batched")
        return self.out, self.stats

    def tune(self, cache_path=None):
        best = L.SdBatchConfig()
        path = None if cache_path is None else str(cache_path).encode()
        L.check(L.lib().sd_dp_psf_trace_batched_tune(
            self.handles, len(self.lenses), ctypes.byref(self.sen), _ptr(self.req_dev),
            self.n_req, ctypes.byref(self.opts), _ptr(self.out), self.total, _ptr(self.stats),
            _ptr(self.ws), self.ws.numel(), _stream(), path, ctypes.byref(best)),
            "sd_dp_psf_trace_batched_tune")
        self.config = best
        return (best.threads, best.rays_per_item, best.blocks_per_sm)


HIT_FIELDS = ("x", "y", "dx", "dy", "dz", "state", "side", "pixel")


def trace_hits(lens: Lens, sensor: DPSensor, req, device="cuda"):
    """Per-ray records of one request (structured numpy element)."""
    q = np.zeros(1, dtype=L.REQUEST_DTYPE)
    for f in ("h_mm", "depth_mm", "lambda_nm", "n_grid", "ks"):
        q[f] = req[f]
    if "v_mm" in req.dtype.names:
        q["v_mm"] = req["v_mm"]
    n = int(req["n_grid"])
    rec = torch.zeros((n * n, 8), dtype=torch.float32, device=device)
    cnt = torch.zeros(1, dtype=torch.int32, device=device)
    sen = sensor.c()
    opts = L.SdTraceOpts(0, 0, 0, 0, int(req["ks"]), n)
    L.check(L.lib().sd_dp_trace_hits(lens.handle, ctypes.byref(sen),
                                     q.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opts),
                                     _ptr(rec), n * n, _ptr(cnt), _stream()),
            "sd_dp_trace_hits")
    k = int(cnt.item())
    rec = rec[:k]
    return {f: rec[:, j] for j, f in enumerate(HIT_FIELDS)}


SD_FIELD_RADIAL, SD_FIELD_QUADRANT = 0, 1


class BankLayout:
    """Bank [F][Z][NL][2][ks][ks] description for the renderer; with
    field_mode=SD_FIELD_QUADRANT a first-quadrant 2-D grid of field points,
    [F][F][Z][NL][2][ks][ks] (x index, y index, both at field_h_mm), used
    through the PSF's flip symmetry about both axes (sd_dp_render only)."""

    def __init__(self, field_h_mm, depths_m, n_lambda, ks, pitch_mm, dtype=torch.float32,
                 field_mode=SD_FIELD_RADIAL):
        self.fh = np.ascontiguousarray(field_h_mm, dtype=np.float32)
        self.dm = np.ascontiguousarray(depths_m, dtype=np.float32)
        self.n_lambda, self.ks, self.pitch_mm, self.dtype = n_lambda, ks, pitch_mm, dtype
        self.field_mode = field_mode

    def c(self):
        return L.SdBankLayout(len(self.fh), len(self.dm), self.n_lambda, self.ks,
                              _DT[self.dtype], self.field_mode,
                              self.fh.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                              self.dm.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                              float(self.pitch_mm), 0.0)

    def shape(self):
        cells = len(self.fh) ** 2 if self.field_mode == SD_FIELD_QUADRANT else len(self.fh)
        return (cells, len(self.dm), self.n_lambda, 2, self.ks, self.ks)


def dp_render(aif, depth_m, bank, layout: BankLayout, out=None):
    """aif (N,C,H,W) f32/bf16/f16, depth (N,H,W) f32 metres, bank in
    layout.dtype -> DP image (N,2C,H,W) in aif's dtype."""
    N, C, H, W = aif.shape
    if out is None:
        out = torch.empty((N, 2 * C, H, W), dtype=aif.dtype, device=aif.device)
    _need_cuda(aif, depth_m, bank, out)
    if bank.dtype != layout.dtype or depth_m.dtype != torch.float32:
        raise ValueError("bank dtype must match the layout; depth must be float32")
    lay = layout.c()
    L.check(L.lib().sd_dp_render(_ptr(aif), _ptr(depth_m), _ptr(bank), ctypes.byref(lay),
                                 N, C, H, W, _DT[aif.dtype], _ptr(out), _stream()),
            "sd_dp_render")
    return out


def render_tc_workspace(layout: BankLayout):
    """Device workspace bytes of dp_render_tc for this bank layout: the error
    flag header and the per-call BF16 re-layout of the bank."""
    n = ctypes.c_size_t(0)
    lay = layout.c()
    L.check(L.lib().sd_dp_render_tc_workspace(ctypes.byref(lay), ctypes.byref(n)),
            "sd_dp_render_tc_workspace")
    return n.value


def dp_render_tc(aif, depth_m, bank, layout: BankLayout, out=None, workspace=None):
    """dp_render of a 16-bit image on the tensor cores: aif (N,C,H,W) bf16
    or f16, depth (N,H,W) f32, bank in aif's dtype (or f32, rounded) ->
    (N,2C,H,W) in aif's dtype.  The workspace's first int32 is an error flag
    (1 = a completion wait gave up)."""
    N, C, H, W = aif.shape
    if aif.dtype not in (torch.bfloat16, torch.float16):
        raise ValueError("the tensor-core render takes a bfloat16 or float16 image")
    if out is None:
        out = torch.empty((N, 2 * C, H, W), dtype=aif.dtype, device=aif.device)
    if workspace is None:
        workspace = torch.empty(render_tc_workspace(layout), dtype=torch.uint8, device=aif.device)
    _need_cuda(aif, depth_m, bank, out, workspace)
    if bank.dtype != layout.dtype or depth_m.dtype != torch.float32:
        raise ValueError("bank dtype must match the layout; depth must be float32")
    lay = layout.c()
    L.check(L.lib().sd_dp_render_tc(_ptr(aif), _ptr(depth_m), _ptr(bank), ctypes.byref(lay),
                                    N, C, H, W, _DT[aif.dtype], _ptr(out), _ptr(workspace),
                                    workspace.numel(), _stream()), "sd_dp_render_tc")
    return out


def render_backward_workspace(layout: BankLayout, N, C, H, W):
    """Device workspace bytes of dp_render_backward: the per-pixel slice
    selection both gradients read, the image gradient's re-laid bank and row
    extents, then the bank gradient's per-tile slice bitmap, its per-slice
    tile counts and launch order (and a quadrant bank's per-flip-class
    gradient slab)."""
    n = ctypes.c_size_t(0)
    lay = layout.c()
    L.check(L.lib().sd_dp_render_backward_workspace(ctypes.byref(lay), N, C, H, W,
                                                    ctypes.byref(n)),
            "sd_dp_render_backward_workspace")
    return n.value


def bank_grad_tc_workspace(layout: BankLayout, N, C, H, W):
    """Device workspace bytes of dp_render_bank_grad_tc: the error flag header,
    the per-pixel slice selection, the per-tile slice bitmap, the per-slice
    tile counts and launch order (and a quadrant bank's per-key slab)."""
    n = ctypes.c_size_t(0)
    lay = layout.c()
    L.check(L.lib().sd_dp_render_bank_grad_tc_workspace(ctypes.byref(lay), N, C, H, W,
                                                        ctypes.byref(n)),
            "sd_dp_render_bank_grad_tc_workspace")
    return n.value


def dp_render_bank_grad_tc(grad_out, aif, depth_m, layout: BankLayout, out=None, workspace=None):
    """Bank gradient of dp_render on the tensor cores: grad_out (N,2C,H,W)
    f32, aif (N,C,H,W) bf16 or f16, depth (N,H,W) f32 -> grad_bank
    (layout.shape()) f32.  The workspace's first int32 is an error flag (1 =
    a completion wait gave up)."""
    N, C, H, W = aif.shape
    if aif.dtype not in (torch.bfloat16, torch.float16) or grad_out.dtype != torch.float32:
        raise ValueError("bf16 or f16 image and float32 output gradient")
    if out is None:
        out = torch.empty(layout.shape(), dtype=torch.float32, device=aif.device)
    if workspace is None:
        workspace = torch.empty(bank_grad_tc_workspace(layout, N, C, H, W), dtype=torch.uint8,
                                device=aif.device)
    _need_cuda(grad_out, aif, depth_m, out, workspace)
    lay = layout.c()
    L.check(L.lib().sd_dp_render_bank_grad_tc(_ptr(grad_out), _ptr(aif), _ptr(depth_m),
                                              ctypes.byref(lay), N, C, H, W, _DT[aif.dtype],
                                              _ptr(out),
                                              _ptr(workspace), workspace.numel(), _stream()),
            "sd_dp_render_bank_grad_tc")
    return out


def dp_render_backward(grad_out, aif, depth_m, bank, layout: BankLayout, need_aif=True,
                       need_bank=True, workspace=None):
    """Adjoint of dp_render: (grad_aif or None, grad_bank or None), both FP32;
    aif and bank may be stored in any dtype dp_render takes."""
    N, C, H, W = aif.shape
    dev = aif.device
    ga = torch.empty(aif.shape, dtype=torch.float32, device=dev) if need_aif else None
    gb = torch.empty(bank.shape, dtype=torch.float32, device=dev) if need_bank else None
    if (need_bank or need_aif) and workspace is None:
        nbytes = render_backward_workspace(layout, N, C, H, W)
        workspace = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
    _need_cuda(grad_out, aif, depth_m, bank, ga, gb)
    if grad_out.dtype != torch.float32 or bank.dtype != layout.dtype:
        raise ValueError("grad_out must be float32 and the bank dtype must match the layout")
    lay = layout.c()
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    L.check(L.lib().sd_dp_render_backward(_ptr(grad_out), _ptr(aif), _ptr(depth_m), _ptr(bank),
                                          ctypes.byref(lay), N, C, H, W, _DT[aif.dtype],
                                          _ptr(ga), _ptr(gb), _ptr(workspace), ws_bytes,
                                          _stream()),
            "sd_dp_render_backward")
    return ga, gb


MLP_HIDDEN = 512
def MLP_SHAPES(ks):
    """(out, in) of the six weight matrices for kernel size ks."""
    return [(MLP_HIDDEN, 3)] + [(MLP_HIDDEN, MLP_HIDDEN)] * 4 + [(2 * ks * ks, MLP_HIDDEN)]


class PsfMLP:
    """The DP PSF prediction network (Sec. 3.2) packed on the device: weights
    [l] (out, in) and biases[l] for l = 0..5 as float arrays of the shapes
    MLP_SHAPES(ks) (3 -> 512, four 512 -> 512, 512 -> 2 ks^2)."""

    def __init__(self, weights, biases, ks, device=None):
        shapes = MLP_SHAPES(ks)
        if len(weights) != 6 or len(biases) != 6:
            raise ValueError("six weight matrices and six bias vectors")
        self.w = [np.ascontiguousarray(w, dtype=np.float32) for w in weights]
        self.b = [np.ascontiguousarray(b, dtype=np.float32) for b in biases]
        for w, b, sh in zip(self.w, self.b, shapes):
            if w.shape != sh or b.shape != (sh[0],):
                raise ValueError(f"layer shapes must be {shapes}")
        self.ks = ks
        n = ctypes.c_size_t(0)
        L.check(L.lib().sd_mlp_blob_bytes(ks, ctypes.byref(n)), "sd_mlp_blob_bytes")
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.blob = torch.empty(n.value, dtype=torch.uint8, device=dev)
        FP = ctypes.POINTER(ctypes.c_float)
        wp = (FP * 6)(*[w.ctypes.data_as(FP) for w in self.w])
        bp = (FP * 6)(*[b.ctypes.data_as(FP) for b in self.b])
        L.check(L.lib().sd_mlp_pack(wp, bp, ks, _ptr(self.blob), self.blob.numel()),
                "sd_mlp_pack")


def mlp_psf_map(net: PsfMLP, depth_m, d_min_m, d_max_m, out=None, status=None,
                dtype=torch.float32):
    """Per-pixel DP PSF map (H, W, 2, ks, ks) in dtype (float32 or bfloat16)
    predicted by the network for a depth map (H, W) in metres (device,
    FP32); returns (map, status) with status a device int32 (1 if a bounded
    wait of the kernel gave up)."""
    H, W = depth_m.shape
    ks = net.ks
    if out is None:
        out = torch.empty((H, W, 2, ks, ks), dtype=dtype, device=depth_m.device)
    if status is None:
        status = torch.empty(1, dtype=torch.int32, device=depth_m.device)
    _need_cuda(depth_m, out, status, net.blob)
    if depth_m.dtype != torch.float32:
        raise ValueError("depth must be float32")
    L.check(L.lib().sd_mlp_psf_map(_ptr(net.blob), ks, _ptr(depth_m), H, W, float(d_min_m),
                                   float(d_max_m), _ptr(out), _DT[out.dtype], _ptr(status),
                                   _stream()), "sd_mlp_psf_map")
    return out, status


def sync_status(status_word):
    """Waits for the current stream and raises SdError (SD_ERR_TIMEOUT) when
    the device status word -- the first int32 of a tensor-core render or
    bank-gradient workspace, or the network's status buffer -- reports that a
    bounded completion wait gave up."""
    _need_cuda(status_word)
    L.check(L.lib().sd_sync_status(_ptr(status_word), _stream()), "device status")


def set_wait_limit(polls):
    """Failure injection for tests: every bounded completion wait of the
    tensor-core kernels launched afterwards gives up after `polls` polls
    (0: at the first wait, before anything asynchronous is issued); None or
    a negative value restores each kernel's own limit."""
    L.check(L.lib().sd_set_wait_limit(-1 if polls is None else int(polls)), "sd_set_wait_limit")


def fp32_peak_launch(sink, blocks, iters):
    """Launches the FP32 throughput probe on the current stream:
    blocks * 256 threads x iters iterations x 32 flops (16 FMA chains)."""
    _need_cuda(sink)
    if sink.numel() < blocks * 256:
        raise ValueError("sink must hold blocks * 256 floats")
    L.check(L.lib().sd_dev_fp32_peak(_ptr(sink), int(blocks), int(iters), _stream()),
            "sd_dev_fp32_peak")
    return float(blocks) * 256 * iters * 32
