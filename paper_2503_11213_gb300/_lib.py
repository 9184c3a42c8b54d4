"""ctypes declarations of the C ABI in include/sdirt.h (marshalling only).

Loading fails loudly when libsdirt.so is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import numpy as np

# the checked build (bounds-checked kernels, sd_check_status) when the
# environment sets SDIRT_CHECKED=1
_LIB_PATH = Path(__file__).resolve().parent / (
    "_build_checked/libsdirt_checked.so" if os.environ.get("SDIRT_CHECKED") == "1"
    else "_build/libsdirt.so")

(SD_OK, SD_ERR_ARG, SD_ERR_LENS, SD_ERR_UNSUPPORTED, SD_ERR_CUDA, SD_ERR_CAPACITY,
 SD_ERR_TIMEOUT) = range(7)
SD_SURF_REFRACT, SD_SURF_STOP = 0, 1
SD_BIN_HARD, SD_BIN_BILINEAR = 0, 1
SD_NORM_NONE, SD_NORM_JOINT, SD_NORM_SEPARATE, SD_NORM_PER_RAY = range(4)
SD_F32, SD_BF16, SD_F16 = 0, 1, 2
SD_N_STATS = 8
SD_MAX_SURFACES = 32
SD_MAX_LENSES = 16
NPAR_SURF = 8                      # curvature, conic, a4..a12, thickness


class SdSurface(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("radius", ctypes.c_double), ("thickness", ctypes.c_double),
                ("nd", ctypes.c_double), ("vd", ctypes.c_double),
                ("semi_diameter", ctypes.c_double), ("conic", ctypes.c_double),
                ("asph", ctypes.c_double * 5)]


class SdParaxial(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("efl", "bfl", "z_ep", "r_ep", "sensor_dist", "m_sensor", "img_dist", "z_sensor")]


class SdSensor(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("pitch_mm", "h_mm", "f_mm", "w_mm", "r_mm")]


class SdTraceOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("norm", ctypes.c_int32),
                ("out_dtype", ctypes.c_int32), ("newton_iters", ctypes.c_int32),
                ("max_ks", ctypes.c_int32), ("max_n_grid", ctypes.c_int32),
                ("land_mask", ctypes.c_void_p)]


class SdBankLayout(ctypes.Structure):
    _fields_ = [("n_field", ctypes.c_int32), ("n_depth", ctypes.c_int32),
                ("n_lambda", ctypes.c_int32), ("ks", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("field_mode", ctypes.c_int32),
                ("field_h_mm", ctypes.POINTER(ctypes.c_float)),
                ("depths_m", ctypes.POINTER(ctypes.c_float)),
                ("pitch_mm", ctypes.c_float), ("reserved2", ctypes.c_float)]


class SdBatchConfig(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("rays_per_item", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# sd_psf_request as a numpy record (56 bytes, device-resident array)
REQUEST_DTYPE = np.dtype([("h_mm", "<f8"), ("depth_mm", "<f8"), ("lambda_nm", "<f8"),
                          ("n_grid", "<i4"), ("ks", "<i4"), ("lens", "<i4"),
                          ("reserved", "<i4"), ("out_offset", "<i8"), ("v_mm", "<f8")])
assert REQUEST_DTYPE.itemsize == 56

# every exported symbol of include/sdirt.h
EXPORTS = ("sd_lens_load", "sd_lens_paraxial", "sd_lens_set_param", "sd_lens_free",
           "sd_dp_psf_trace", "sd_dp_psf_trace_backward", "sd_dp_psf_trace_mask_bytes",
           "sd_dp_psf_trace_batched",
           "sd_dp_psf_trace_batched_workspace", "sd_dp_psf_trace_batched_tune",
           "sd_dp_trace_hits", "sd_dp_psf_map",
           "sd_dp_render", "sd_dp_render_map", "sd_dp_render_tc", "sd_dp_render_tc_workspace", "sd_dp_render_backward",
           "sd_dp_render_backward_workspace", "sd_dp_render_backward_noalloc",
           "sd_mlp_blob_bytes", "sd_mlp_pack", "sd_mlp_psf_map",
           "sd_dp_render_bank_grad_tc", "sd_dp_render_bank_grad_tc_workspace",
           "sd_dev_math_check", "sd_dev_tc_check", "sd_status_string", "sd_last_cuda_error",
           "sd_version", "sd_sync_status", "sd_set_wait_limit", "sd_dev_fp32_peak",
           "sd_check_status")

_lib = None


class SdError(RuntimeError):
    def __init__(self, status, what):
        name = lib().sd_status_string(status).decode() if _lib else str(status)
        extra = ""
        if status == SD_ERR_CUDA and _lib:
            extra = f" (cudaError {_lib.sd_last_cuda_error()})"
        super().__init__(f"{what}: {name}{extra}")
        self.status = status


def check(status, what):
    if status != SD_OK:
        raise SdError(status, what)


def lib():
    """Loads libsdirt.so (build it with paper_2503_11213_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise RuntimeError(f"sdirt CUDA library not built: {_LIB_PATH} is missing "
                           "(run paper_2503_11213_gb300.build.build()); there is no "
                           "CPU fallback")
    import torch  # noqa: F401  -- load the CUDA runtime torch uses first
    L = ctypes.CDLL(str(_LIB_PATH))
    P = ctypes.POINTER
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.sd_lens_load.argtypes = [P(SdSurface), i32, dbl, P(vp)]
    L.sd_lens_paraxial.argtypes = [vp, dbl, dbl, P(SdParaxial)]
    L.sd_lens_set_param.argtypes = [vp, i32, dbl]
    L.sd_lens_free.argtypes = [vp]
    L.sd_dp_psf_trace.argtypes = [P(vp), i32, P(SdSensor), vp, i32, P(SdTraceOpts), vp, vp, vp]
    L.sd_dp_psf_trace_backward.argtypes = [P(vp), i32, P(SdSensor), vp, i32, P(SdTraceOpts),
                                           vp, vp, vp, vp, vp]
    L.sd_dp_psf_trace_mask_bytes.argtypes = [i32, i32, P(ctypes.c_size_t)]
    L.sd_check_status.argtypes = [P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32),
                                  P(ctypes.c_int64)]
    ll = ctypes.c_longlong
    L.sd_dp_psf_trace_batched_workspace.argtypes = [i32, ll, P(ctypes.c_size_t)]
    L.sd_dp_psf_trace_batched.argtypes = [P(vp), i32, P(SdSensor), vp, i32, P(SdTraceOpts),
                                          P(SdBatchConfig), vp, ll, vp, vp, ctypes.c_size_t, vp]
    L.sd_dp_psf_trace_batched_tune.argtypes = [P(vp), i32, P(SdSensor), vp, i32, P(SdTraceOpts),
                                               vp, ll, vp, vp, ctypes.c_size_t, vp,
                                               ctypes.c_char_p, P(SdBatchConfig)]
    L.sd_dp_trace_hits.argtypes = [vp, P(SdSensor), vp, P(SdTraceOpts), vp, i32, vp, vp]
    L.sd_dp_psf_map.argtypes = [vp, P(SdSensor), vp, i32, i32, dbl, i32, i32, P(SdTraceOpts),
                                vp, vp, vp]
    L.sd_dp_render_tc.argtypes = [vp, vp, vp, P(SdBankLayout), i32, i32, i32, i32, i32, vp, vp,
                                  ctypes.c_size_t, vp]
    L.sd_dp_render_tc_workspace.argtypes = [P(SdBankLayout), P(ctypes.c_size_t)]
    L.sd_dp_render_map.argtypes = [vp, vp, i32, i32, i32, i32, i32, i32, i32, vp, vp, vp]
    L.sd_dp_render.argtypes = [vp, vp, vp, P(SdBankLayout), i32, i32, i32, i32, i32, vp, vp]
    L.sd_dp_render_backward.argtypes = [vp, vp, vp, vp, P(SdBankLayout), i32, i32, i32, i32,
                                        i32, vp, vp, vp, ctypes.c_size_t, vp]
    L.sd_dp_render_backward_noalloc.argtypes = [vp, vp, vp, vp, P(SdBankLayout), i32, i32, i32,
                                                 i32, vp, vp, vp]
    L.sd_dp_render_backward_workspace.argtypes = [P(SdBankLayout), i32, i32, i32, i32,
                                                  P(ctypes.c_size_t)]
    L.sd_dev_math_check.argtypes = [vp, vp, i32, vp, vp, vp]
    L.sd_dev_tc_check.argtypes = [vp, vp, i32, vp, vp, vp]
    L.sd_dp_render_bank_grad_tc_workspace.argtypes = [P(SdBankLayout), i32, i32, i32, i32,
                                                      P(ctypes.c_size_t)]
    L.sd_dp_render_bank_grad_tc.argtypes = [vp, vp, vp, P(SdBankLayout), i32, i32, i32, i32, i32,
                                            vp, vp, ctypes.c_size_t, vp]
    fl = ctypes.c_float
    L.sd_mlp_blob_bytes.argtypes = [i32, P(ctypes.c_size_t)]
    L.sd_mlp_pack.argtypes = [P(P(fl)), P(P(fl)), i32, vp, ctypes.c_size_t]
    L.sd_mlp_psf_map.argtypes = [vp, i32, vp, i32, i32, fl, fl, vp, i32, vp, vp]
    L.sd_sync_status.argtypes = [vp, vp]
    L.sd_set_wait_limit.argtypes = [ll]
    L.sd_dev_fp32_peak.argtypes = [vp, i32, i32, vp]
    L.sd_status_string.argtypes = [i32]
    L.sd_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "sd_status_string":
            getattr(L, name).restype = i32
    _lib = L
    return L
