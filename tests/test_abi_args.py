"""Argument checks that the render, network and backward entry points make
on the host before any CUDA call (include/sdirt.h: "Argument errors are
reported synchronously before anything is launched").  The pointers passed
are host placeholders that no call may dereference, so the module runs only
where no CUDA device exists (a check that wrongly passed would otherwise
launch a kernel on them)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2503_11213_gb300 import _lib as L
from paper_2503_11213_gb300 import build as B

pytestmark = pytest.mark.skipif(torch.cuda.is_available(),
                                reason="host placeholders as device pointers: CPU only")

_BUF = ctypes.create_string_buffer(4096)
PTR = ctypes.cast(_BUF, ctypes.c_void_p)                     # 16-byte aligned or better
MIS = ctypes.c_void_p(ctypes.addressof(_BUF) + 8)            # not 256-byte aligned
ALIGNED = ctypes.c_void_p((ctypes.addressof(_BUF) + 255) // 256 * 256)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def layout(ks=65, nl=3, dtype=L.SD_F32, nf=3, nz=3):
    fh = np.linspace(0.0, 1.0, nf).astype(np.float32)
    dm = np.linspace(0.5, 3.0, nz).astype(np.float32)
    lay = L.SdBankLayout(nf, nz, nl, ks, dtype, 0,
                         fh.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                         dm.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 0.002, 0.0)
    return lay, (fh, dm)


def test_render_map_args(lib):
    f = lib.sd_dp_render_map
    F32, BF16, F16 = L.SD_F32, L.SD_BF16, L.SD_F16
    assert f(None, PTR, 1, 3, 8, 8, 5, F32, F32, PTR, None, None) == L.SD_ERR_ARG
    assert f(PTR, PTR, 1, 3, 8, 8, 4, F32, F32, PTR, None, None) == L.SD_ERR_ARG      # even ks
    assert f(PTR, PTR, 1, 0, 8, 8, 5, F32, F32, PTR, None, None) == L.SD_ERR_ARG      # C < 1
    assert f(PTR, PTR, -1, 3, 8, 8, 5, F32, F32, PTR, None, None) == L.SD_ERR_ARG
    assert f(PTR, PTR, 1, 3, 8, 8, 129, F32, F32, PTR, None, None) == L.SD_ERR_UNSUPPORTED
    assert f(PTR, PTR, 70000, 1, 8, 8, 5, F32, F32, PTR, None, None) == L.SD_ERR_UNSUPPORTED
    # image / map storage pairs outside the supported set
    assert f(PTR, PTR, 1, 3, 8, 8, 5, BF16, F32, PTR, None, None) == L.SD_ERR_UNSUPPORTED
    assert f(PTR, PTR, 1, 3, 8, 8, 5, F16, BF16, PTR, None, None) == L.SD_ERR_UNSUPPORTED
    # empty inputs: nothing to do
    assert f(PTR, PTR, 0, 3, 8, 8, 5, F32, F32, PTR, None, None) == L.SD_OK
    assert f(PTR, PTR, 1, 3, 0, 8, 5, F32, F32, PTR, None, None) == L.SD_OK


def test_render_args(lib):
    lay, keep = layout()
    f = lib.sd_dp_render
    assert f(None, PTR, PTR, ctypes.byref(lay), 1, 3, 8, 8, L.SD_F32, PTR, None) == L.SD_ERR_ARG
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 0, 8, 8, L.SD_F32, PTR, None) == L.SD_ERR_ARG
    # C must equal n_lambda (3) or n_lambda must be 1
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 2, 8, 8, L.SD_F32, PTR, None) == L.SD_ERR_ARG
    # storage pairs outside the supported set (image F16 with an F32 bank)
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 8, 8, L.SD_F16, PTR, None) == \
        L.SD_ERR_UNSUPPORTED
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 0, 3, 8, 8, L.SD_F32, PTR, None) == L.SD_OK
    big, keep2 = layout(nf=256, nz=256)    # 65,536 slice keys: more than 16-bit keys hold
    assert f(PTR, PTR, PTR, ctypes.byref(big), 1, 3, 8, 8, L.SD_F32, PTR, None) == \
        L.SD_ERR_UNSUPPORTED


def test_render_tc_args(lib):
    lay, keep = layout(dtype=L.SD_BF16)
    n = ctypes.c_size_t(0)
    assert lib.sd_dp_render_tc_workspace(ctypes.byref(lay), ctypes.byref(n)) == L.SD_OK
    f = lib.sd_dp_render_tc
    ws = n.value
    BF = L.SD_BF16
    # the workspace: missing, short or not 256-byte aligned
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 8, 8, BF, PTR, None, ws, None) == L.SD_ERR_ARG
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 8, 8, BF, PTR, ALIGNED, ws - 1, None) == \
        L.SD_ERR_ARG
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 8, 8, BF, PTR, MIS, ws, None) == L.SD_ERR_ARG
    # ks above 65, an FP32 image and a bank of the other 16-bit type are not
    # supported on the tensor cores (both operands of a product share a type)
    lay67, keep67 = layout(ks=67, dtype=L.SD_BF16)
    assert f(PTR, PTR, PTR, ctypes.byref(lay67), 1, 3, 8, 8, BF, PTR, ALIGNED, 1 << 40, None) == \
        L.SD_ERR_UNSUPPORTED
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 8, 8, L.SD_F32, PTR, ALIGNED, 1 << 40,
             None) == L.SD_ERR_UNSUPPORTED
    lay16, keep16 = layout(dtype=L.SD_F16)
    assert f(PTR, PTR, PTR, ctypes.byref(lay16), 1, 3, 8, 8, BF, PTR, ALIGNED, 1 << 40, None) == \
        L.SD_ERR_UNSUPPORTED
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 8, 8, L.SD_F16, PTR, ALIGNED, 1 << 40,
             None) == L.SD_ERR_UNSUPPORTED
    # empty inputs after a valid workspace: nothing to do (BF16, FP16, and
    # an FP32 bank rounded to either)
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 0, 3, 8, 8, BF, PTR, ALIGNED, ws, None) == L.SD_OK
    assert f(PTR, PTR, PTR, ctypes.byref(lay16), 0, 3, 8, 8, L.SD_F16, PTR, ALIGNED, ws,
             None) == L.SD_OK
    lay32, keep32 = layout(dtype=L.SD_F32)
    assert f(PTR, PTR, PTR, ctypes.byref(lay32), 0, 3, 8, 8, L.SD_F16, PTR, ALIGNED, 1 << 40,
             None) == L.SD_OK


def test_render_backward_args(lib):
    lay, keep = layout()
    f = lib.sd_dp_render_backward
    args = lambda dt, ga, gb, ws, nb: (PTR, PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 64, 64, dt,
                                       ga, gb, ws, nb, None)
    assert f(None, PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 64, 64, L.SD_F32, PTR, PTR, PTR, 0,
             None) == L.SD_ERR_ARG
    assert f(*args(7, PTR, None, None, 0)) == L.SD_ERR_UNSUPPORTED      # image dtype
    # the bank gradient needs at least the selection table and the tile
    # bitmap in the workspace
    assert f(*args(L.SD_F32, None, PTR, None, 0)) == L.SD_ERR_ARG
    assert f(*args(L.SD_F32, None, PTR, PTR, 4)) == L.SD_ERR_ARG
    # the image gradient needs the selection table and its own (re-laid
    # bank, row extents) in a 256-byte aligned workspace
    assert f(*args(L.SD_F32, PTR, None, None, 0)) == L.SD_ERR_ARG
    assert f(*args(L.SD_F32, PTR, None, ALIGNED, 4096)) == L.SD_ERR_ARG
    assert f(*args(L.SD_F32, PTR, None, MIS, 1 << 40)) == L.SD_ERR_ARG


def test_bank_grad_tc_args(lib):
    lay, keep = layout(dtype=L.SD_BF16)
    n = ctypes.c_size_t(0)
    assert lib.sd_dp_render_bank_grad_tc_workspace(ctypes.byref(lay), 1, 3, 64, 64,
                                                   ctypes.byref(n)) == L.SD_OK
    f = lib.sd_dp_render_bank_grad_tc
    BF = L.SD_BF16
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 64, 64, BF, None, ALIGNED, n.value, None) == \
        L.SD_ERR_ARG                                                     # no grad_bank
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 64, 64, BF, PTR, MIS, n.value, None) == \
        L.SD_ERR_ARG                                                     # misaligned
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 64, 64, BF, PTR, ALIGNED, 16, None) == \
        L.SD_ERR_ARG                                                     # short
    lay67, keep67 = layout(ks=67, dtype=L.SD_BF16)
    assert f(PTR, PTR, PTR, ctypes.byref(lay67), 1, 3, 64, 64, BF, PTR, ALIGNED, 1 << 40,
             None) == L.SD_ERR_UNSUPPORTED                               # ks > 65
    assert f(PTR, PTR, PTR, ctypes.byref(lay), 1, 3, 64, 64, L.SD_F32, PTR, ALIGNED, 1 << 40,
             None) == L.SD_ERR_UNSUPPORTED                               # FP32 image


def test_mlp_map_args(lib):
    f = lib.sd_mlp_psf_map
    ok = (ALIGNED, 21, PTR, 8, 8, 0.5, 20.0, PTR, L.SD_F32, PTR, None)

    def call(**kw):
        a = list(ok)
        names = ["blob", "ks", "depth", "H", "W", "dmin", "dmax", "out", "dt", "status", "s"]
        for k, v in kw.items():
            a[names.index(k)] = v
        return f(*a)

    assert call(blob=None) == L.SD_ERR_ARG
    assert call(status=None) == L.SD_ERR_ARG
    assert call(ks=20) == L.SD_ERR_ARG
    assert call(ks=33) == L.SD_ERR_ARG
    assert call(H=0) == L.SD_ERR_ARG
    assert call(W=-2) == L.SD_ERR_ARG
    assert call(dmin=3.0, dmax=3.0) == L.SD_ERR_ARG
    assert call(dmax=float("nan")) == L.SD_ERR_ARG
    assert call(dt=L.SD_F16) == L.SD_ERR_UNSUPPORTED
    assert call(blob=MIS) == L.SD_ERR_ARG


def test_check_status_needs_the_checked_build(lib):
    # the normal build compiles its bounds checks away and says so before
    # touching the device
    site, index, bound = ctypes.c_int32(7), ctypes.c_int32(0), ctypes.c_int32(0)
    count = ctypes.c_int64(7)
    assert lib.sd_check_status(ctypes.byref(site), ctypes.byref(index), ctypes.byref(bound),
                               ctypes.byref(count)) == L.SD_ERR_UNSUPPORTED
    assert lib.sd_check_status(None, None, None, ctypes.byref(count)) == L.SD_ERR_ARG
    assert lib.sd_check_status(ctypes.byref(site), None, None, None) == L.SD_ERR_ARG
