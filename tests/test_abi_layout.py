"""Host-side validation of the bank layout (include/sdirt.h, "Every call
that takes a layout validates it on the host before any CUDA call") and the
workspace queries, through calls that need no GPU."""
import ctypes

import numpy as np
import pytest

import paper_2503_11213_gb300 as sd
from paper_2503_11213_gb300 import _lib as L
from paper_2503_11213_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def layout(fh=(0.0, 0.5, 1.0), dm=(0.5, 1.0, 3.0), nl=3, ks=65, pitch=0.002, mode=0,
           dtype=L.SD_BF16):
    fh = np.ascontiguousarray(fh, dtype=np.float32)
    dm = np.ascontiguousarray(dm, dtype=np.float32)
    lay = L.SdBankLayout(len(fh), len(dm), nl, ks, dtype, mode,
                         fh.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                         dm.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), pitch, 0.0)
    return lay, (fh, dm)  # keep the arrays alive with the struct


def tc_ws(lib, lay):
    n = ctypes.c_size_t(0)
    return lib.sd_dp_render_tc_workspace(ctypes.byref(lay), ctypes.byref(n)), n.value


def bwd_ws(lib, lay, N=1, C=3, H=64, W=64):
    n = ctypes.c_size_t(0)
    return lib.sd_dp_render_backward_workspace(ctypes.byref(lay), N, C, H, W,
                                               ctypes.byref(n)), n.value


def bg_ws(lib, lay, N=1, C=3, H=64, W=64):
    n = ctypes.c_size_t(0)
    return lib.sd_dp_render_bank_grad_tc_workspace(ctypes.byref(lay), N, C, H, W,
                                                   ctypes.byref(n)), n.value


def test_valid_layouts_accepted(lib):
    for mode in (0, 1):
        lay, keep = layout(mode=mode)
        for q in (tc_ws, bwd_ws, bg_ws):
            st, n = q(lib, lay)
            assert st == L.SD_OK and n > 0


@pytest.mark.parametrize("kw,status", [
    (dict(ks=64), L.SD_ERR_ARG),
    (dict(ks=0), L.SD_ERR_ARG),
    (dict(ks=-3), L.SD_ERR_ARG),
    (dict(ks=129), L.SD_ERR_UNSUPPORTED),
    (dict(nl=0), L.SD_ERR_ARG),
    (dict(pitch=0.0), L.SD_ERR_ARG),
    (dict(pitch=-0.002), L.SD_ERR_ARG),
    (dict(pitch=float("nan")), L.SD_ERR_ARG),
    (dict(fh=(0.0, 0.5, 0.5)), L.SD_ERR_ARG),
    (dict(fh=(0.0, 1.0, 0.5)), L.SD_ERR_ARG),
    (dict(dm=(0.5, 0.5, 3.0)), L.SD_ERR_ARG),
    (dict(dm=(3.0, 1.0, 0.5)), L.SD_ERR_ARG),
    (dict(dm=(0.0, 1.0, 3.0)), L.SD_ERR_ARG),
    (dict(dm=(-1.0, 1.0, 3.0)), L.SD_ERR_ARG),
    (dict(mode=2), L.SD_ERR_ARG),
    (dict(mode=1, fh=(-0.1, 0.5, 1.0)), L.SD_ERR_ARG),
    (dict(fh=np.linspace(0, 1, 257)), L.SD_ERR_ARG),
    (dict(dm=np.linspace(0.5, 3, 257)), L.SD_ERR_ARG),
])
def test_invalid_layouts_rejected(lib, kw, status):
    lay, keep = layout(**kw)
    for q in (tc_ws, bwd_ws, bg_ws):
        assert q(lib, lay)[0] == status, (q.__name__, kw)


def test_radial_with_negative_first_height_is_valid(lib):
    # only a quadrant grid needs heights >= 0 (it mirrors |X|, |Y|)
    lay, keep = layout(fh=(-0.1, 0.5, 1.0))
    assert tc_ws(lib, lay)[0] == L.SD_OK


def test_null_layout_pointers(lib):
    n = ctypes.c_size_t(0)
    assert lib.sd_dp_render_tc_workspace(None, ctypes.byref(n)) == L.SD_ERR_ARG
    lay, keep = layout()
    lay.field_h_mm = None
    assert tc_ws(lib, lay)[0] == L.SD_ERR_ARG
    lay, keep = layout()
    lay.depths_m = None
    assert tc_ws(lib, lay)[0] == L.SD_ERR_ARG
    lay, keep = layout()
    assert lib.sd_dp_render_tc_workspace(ctypes.byref(lay), None) == L.SD_ERR_ARG


def test_bad_image_sizes_rejected(lib):
    lay, keep = layout()
    assert bwd_ws(lib, lay, N=-1)[0] == L.SD_ERR_ARG
    assert bwd_ws(lib, lay, C=0)[0] == L.SD_ERR_ARG
    assert bwd_ws(lib, lay, H=-5)[0] == L.SD_ERR_ARG
    # C must equal n_lambda or n_lambda must be 1
    assert bwd_ws(lib, lay, C=2)[0] == L.SD_ERR_ARG
    lay1, keep1 = layout(nl=1)
    assert bwd_ws(lib, lay1, C=2)[0] == L.SD_OK


def test_tc_workspace_holds_the_bf16_relayout(lib):
    # a BF16 copy of every tap of every slice the selection can produce (4
    # flip classes for a quadrant bank), after the 256-byte flag header
    for mode, cells in ((0, 3), (1, 9)):
        lay, keep = layout(mode=mode)
        st, n = tc_ws(lib, lay)
        keys = cells * 3 * (4 if mode == 1 else 1)
        assert st == L.SD_OK and n >= 256 + keys * 3 * 2 * 65 * 65 * 2


def test_backward_workspace_holds_selection_image_tables_bitmap_and_plan(lib):
    # an 8-byte selection per pixel (both passes), the image gradient's
    # tables (every key's kernel re-laid as FP32 columns of at least ks rows
    # per side, a 2-byte extent per kernel row), then the bank gradient's
    # tile bitmaps, for a quadrant bank an FP32 gradient slab per key (flip
    # class), and the work plan: 8 bytes per key (tile count, launch order)
    # and two chunk slabs (all wavelengths) for each of max(32, keys / 8)
    # split slices
    N, C, H, W = 2, 3, 100, 130
    for mode, cells in ((0, 3), (1, 9)):
        lay, keep = layout(mode=mode)
        st, n = bwd_ws(lib, lay, N, C, H, W)
        keys = cells * 3 * (4 if mode == 1 else 1)
        tiles = N * -(-H // 32) * -(-W // 64)
        assert st == L.SD_OK
        sel_part = N * H * W * 8
        slab = keys * 3 * 2 * 65 * 65 * 4
        bitmap = tiles * keys // 8
        plan = 8 * keys + 2 * max(32, keys // 8) * 3 * 2 * 65 * 65 * 4
        img_part = keys * 3 * 65 * (65 * 2 * 4 + 2)
        assert n >= sel_part + img_part + bitmap + plan + (slab if mode == 1 else 0)
        # the tensor-core bank gradient needs the same bank-pass parts but no
        # image tables
        st2, n2 = bg_ws(lib, lay, N, C, H, W)
        assert st2 == L.SD_OK and sel_part + bitmap + plan + (slab if mode == 1 else 0) <= n2
        assert n2 < n


def test_workspace_grows_with_the_problem(lib):
    lay, keep = layout()
    small = bwd_ws(lib, lay, 1, 3, 64, 64)[1]
    assert bwd_ws(lib, lay, 4, 3, 64, 64)[1] >= small
    assert bwd_ws(lib, lay, 1, 3, 512, 512)[1] >= small
    big, keep2 = layout(fh=np.linspace(0, 1, 32), dm=np.linspace(0.3, 3, 32))
    assert bwd_ws(lib, big, 1, 3, 64, 64)[1] > small


def test_mlp_blob_bytes(lib):
    n = ctypes.c_size_t(0)
    for ks in (0, -1, 2, 20, 33):
        assert lib.sd_mlp_blob_bytes(ks, ctypes.byref(n)) == L.SD_ERR_ARG
    assert lib.sd_mlp_blob_bytes(21, None) == L.SD_ERR_ARG
    prev = 0
    for ks in (1, 5, 21, 31):
        assert lib.sd_mlp_blob_bytes(ks, ctypes.byref(n)) == L.SD_OK
        # at least the BF16 512-wide matrices and the FP32 layer 0 and biases
        need = 2 * (4 * 512 * 512 + 2 * ks * ks * 512) + 4 * (512 * 4 + 4 * 512 + 2 * ks * ks)
        assert n.value >= need and n.value >= prev
        prev = n.value


def test_batched_workspace(lib):
    n = ctypes.c_size_t(0)
    assert lib.sd_dp_psf_trace_batched_workspace(-1, 10, ctypes.byref(n)) == L.SD_ERR_ARG
    assert lib.sd_dp_psf_trace_batched_workspace(3, -1, ctypes.byref(n)) == L.SD_ERR_ARG
    assert lib.sd_dp_psf_trace_batched_workspace(3, 10, None) == L.SD_ERR_ARG
    assert lib.sd_dp_psf_trace_batched_workspace(0, 0, ctypes.byref(n)) == L.SD_OK
    assert lib.sd_dp_psf_trace_batched_workspace(100, 2 * 65 * 65 * 100, ctypes.byref(n)) == L.SD_OK
    # a 32-bit count per output element of every request
    assert n.value >= 4 * 2 * 65 * 65 * 100


def test_landing_mask_bytes(lib):
    # one bit per pupil sample of the largest grid, whole 32-bit words per
    # request (0 = the 512 default)
    n = ctypes.c_size_t(0)
    assert lib.sd_dp_psf_trace_mask_bytes(3, 96, ctypes.byref(n)) == L.SD_OK
    assert n.value == 3 * 288 * 4
    assert lib.sd_dp_psf_trace_mask_bytes(2, 0, ctypes.byref(n)) == L.SD_OK
    assert n.value == 2 * 512 * 512 // 8
    assert lib.sd_dp_psf_trace_mask_bytes(5, 7, ctypes.byref(n)) == L.SD_OK
    assert n.value == 5 * 2 * 4
    assert lib.sd_dp_psf_trace_mask_bytes(0, 64, ctypes.byref(n)) == L.SD_OK and n.value == 0
    assert lib.sd_dp_psf_trace_mask_bytes(-1, 64, ctypes.byref(n)) == L.SD_ERR_ARG
    assert lib.sd_dp_psf_trace_mask_bytes(1, 4096, ctypes.byref(n)) == L.SD_ERR_ARG
    assert lib.sd_dp_psf_trace_mask_bytes(1, 64, None) == L.SD_ERR_ARG
    # the options struct keeps its size: the mask pointer replaced two
    # reserved words
    assert ctypes.sizeof(L.SdTraceOpts) == 32
