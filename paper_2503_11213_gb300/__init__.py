"""GB300-native (sm_103a) hot path of the Sdirt dual-pixel simulator.

Ray trace of a lens, DP PSF binning and per-pixel DP rendering run in the
CUDA library built from csrc/ (C ABI in include/sdirt.h); this package only
marshals PyTorch tensors into that ABI.
"""
from .api import (SD_FIELD_QUADRANT, SD_FIELD_RADIAL, BankLayout, BatchedTrace, DPSensor, Lens, dp_psf_map, dp_psf_trace,  # noqa: F401
                  dp_psf_trace_backward, dp_render, dp_render_backward, dp_render_map, dp_render_tc,
                  f_number_table, make_requests, render_backward_workspace, trace_hits,
                  PsfMLP, mlp_psf_map, MLP_SHAPES, dp_render_bank_grad_tc, sync_status,
                  set_wait_limit, fp32_peak_launch, land_mask, land_mask_bytes)
from .bank_io import lens_sha256, load_bank, save_bank  # noqa: F401
from .autograd import (DPRenderFunction, DPTraceFunction, dp_psf_trace_autograd,  # noqa: F401
                       dp_render_autograd)
from ._lib import (SD_BF16, SD_BIN_BILINEAR, SD_BIN_HARD, SD_F16, SD_F32, SD_NORM_JOINT,  # noqa: F401
                   SD_NORM_NONE,
                   SD_NORM_PER_RAY, SD_NORM_SEPARATE, SdError, lib)
