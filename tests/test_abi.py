"""The C-ABI library loads and exports every function include/sdirt.h
declares; argument validation that happens before any CUDA call (no GPU)."""
import ctypes
import re
from pathlib import Path

import pytest

import paper_2503_11213_gb300 as sd
from paper_2503_11213_gb300 import _lib as L
from paper_2503_11213_gb300 import build as B

HEADER = Path(__file__).resolve().parents[1] / "include" / "sdirt.h"


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sd_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(L.EXPORTS)


def test_status_strings_and_version(lib):
    assert lib.sd_status_string(L.SD_OK) == b"ok"
    assert lib.sd_status_string(L.SD_ERR_ARG) == b"invalid argument"
    assert lib.sd_status_string(99) == b"unknown status"
    assert lib.sd_version() >= 100


def test_null_arguments_rejected_without_gpu(lib):
    out = ctypes.c_void_p()
    assert lib.sd_lens_load(None, 3, 0.0, ctypes.byref(out)) == L.SD_ERR_ARG
    assert lib.sd_lens_free(None) == L.SD_ERR_ARG
    lay = L.SdBankLayout()
    assert lib.sd_dp_render(None, None, None, ctypes.byref(lay), 1, 1, 8, 8, 0, None,
                            None) == L.SD_ERR_ARG
    opts = L.SdTraceOpts()
    assert lib.sd_dp_psf_trace(None, 0, None, None, 1, ctypes.byref(opts), None, None,
                               None) == L.SD_ERR_ARG


def test_request_record_layout():
    assert L.REQUEST_DTYPE.itemsize == 56
    assert ctypes.sizeof(L.SdSurface) == 8 + 8 * 11
    assert ctypes.sizeof(L.SdTraceOpts) == 32
