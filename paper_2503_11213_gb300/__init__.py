"""GB300-native (sm_103a) hot path of the Sdirt dual-pixel simulator.

Ray trace of a lens, DP PSF binning and per-pixel DP rendering run in the
CUDA library built from csrc/ (C ABI in include/sdirt.h); this package only
marshals PyTorch tensors into that ABI.
"""
from .api import (BankLayout, BatchedTrace, DPSensor, Lens, dp_psf_trace, dp_psf_trace_backward,  # noqa: F401
                  dp_render, dp_render_backward, make_requests, render_backward_workspace,
                  trace_hits)
from ._lib import (SD_BIN_BILINEAR, SD_BIN_HARD, SD_NORM_JOINT, SD_NORM_NONE,  # noqa: F401
                   SD_NORM_PER_RAY, SD_NORM_SEPARATE, SdError, lib)
