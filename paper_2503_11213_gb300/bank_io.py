"""PSF bank files: a traced bank saved with its layout, so that it can be
reused without tracing again (the paper fits its PSF network offline to
traced PSFs, Sec. 3.2).

File layout (little endian):
  8 bytes   magic b"SDBANK" + format version (uint16, 1)
  4 bytes   length of the header (uint32)
  header    UTF-8 JSON: the layout (field heights, depths, wavelength count,
            ks, pixel pitch, field mode, storage dtype), the bank's shape,
            optional provenance (SHA-256 of the lens prescription, the DP
            sensor parameters, the wavelengths), the payload's byte count and
            SHA-256
  payload   the bank's elements in the order [cells][Z][NL][2][ks][ks]
            (FP32, or the 16-bit patterns of BF16 / FP16)

Loading checks the magic, the version, the sizes and the payload hash, and,
when a lens prescription is given, that it is the one the bank was traced
with; any mismatch raises ValueError.
"""
from __future__ import annotations

import dataclasses
import hashlib
import json
import struct

import numpy as np
import torch

from .api import SD_FIELD_QUADRANT, SD_FIELD_RADIAL, BankLayout, DPSensor

MAGIC = b"SDBANK"
VERSION = 1
_DTYPES = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}
_NAMES = {v: k for k, v in _DTYPES.items()}


def lens_sha256(table) -> str:
    """SHA-256 of a lens prescription (the float64 rows ``workloads`` builds)."""
    return hashlib.sha256(np.ascontiguousarray(table, dtype=np.float64).tobytes()).hexdigest()


def _payload(bank: torch.Tensor) -> bytes:
    t = bank.detach().contiguous().cpu().reshape(-1)
    if t.dtype == torch.float32:
        return t.numpy().astype("<f4").tobytes()
    return t.view(torch.int16).numpy().astype("<i2").tobytes()


def save_bank(path, bank: torch.Tensor, layout: BankLayout, lens_table=None,
              sensor: DPSensor | None = None, lambdas_nm=None) -> None:
    """Writes bank (any device, layout.dtype, layout.shape() elements) and its
    layout to path; lens_table / sensor / lambdas_nm are stored as provenance."""
    if bank.dtype != layout.dtype:
        raise ValueError("the bank dtype must match the layout")
    shape = list(layout.shape())
    if bank.numel() != int(np.prod(shape)):
        raise ValueError(f"bank has {bank.numel()} elements, the layout {int(np.prod(shape))}")
    payload = _payload(bank)
    header = {
        "version": VERSION,
        "layout": {"field_h_mm": [float(v) for v in layout.fh],
                   "depths_m": [float(v) for v in layout.dm],
                   "n_lambda": int(layout.n_lambda), "ks": int(layout.ks),
                   "pitch_mm": float(layout.pitch_mm), "field_mode": int(layout.field_mode),
                   "dtype": _NAMES[layout.dtype]},
        "shape": shape,
        "lens_sha256": lens_sha256(lens_table) if lens_table is not None else None,
        "sensor": dataclasses.asdict(sensor) if sensor is not None else None,
        "lambdas_nm": [float(v) for v in lambdas_nm] if lambdas_nm is not None else None,
        "payload_bytes": len(payload),
        "payload_sha256": hashlib.sha256(payload).hexdigest(),
    }
    hb = json.dumps(header, sort_keys=True).encode("utf-8")
    with open(path, "wb") as f:
        f.write(MAGIC + struct.pack("<H", VERSION) + struct.pack("<I", len(hb)))
        f.write(hb)
        f.write(payload)


def load_bank(path, device="cuda", lens_table=None):
    """Reads a bank file: (bank tensor on device, BankLayout, header dict)."""
    with open(path, "rb") as f:
        data = f.read()
    if len(data) < 12 or data[:6] != MAGIC:
        raise ValueError(f"{path}: not a PSF bank file")
    (version,) = struct.unpack("<H", data[6:8])
    if version != VERSION:
        raise ValueError(f"{path}: bank file version {version}, this library reads {VERSION}")
    (hlen,) = struct.unpack("<I", data[8:12])
    if 12 + hlen > len(data):
        raise ValueError(f"{path}: truncated header")
    header = json.loads(data[12:12 + hlen].decode("utf-8"))
    payload = data[12 + hlen:]
    if len(payload) != header["payload_bytes"]:
        raise ValueError(f"{path}: payload has {len(payload)} bytes, the header "
                         f"{header['payload_bytes']}")
    if hashlib.sha256(payload).hexdigest() != header["payload_sha256"]:
        raise ValueError(f"{path}: payload checksum mismatch")
    if lens_table is not None and header["lens_sha256"] != lens_sha256(lens_table):
        raise ValueError(f"{path}: the bank was traced with another lens prescription")
    lay = header["layout"]
    dtype = _DTYPES[lay["dtype"]]
    if lay["field_mode"] not in (SD_FIELD_RADIAL, SD_FIELD_QUADRANT):
        raise ValueError(f"{path}: unknown field mode {lay['field_mode']}")
    layout = BankLayout(np.array(lay["field_h_mm"], dtype=np.float32),
                        np.array(lay["depths_m"], dtype=np.float32), lay["n_lambda"], lay["ks"],
                        lay["pitch_mm"], dtype=dtype, field_mode=lay["field_mode"])
    shape = tuple(layout.shape())
    if list(shape) != header["shape"]:
        raise ValueError(f"{path}: shape {header['shape']} does not match the layout {shape}")
    n = int(np.prod(shape))
    if len(payload) != n * (4 if dtype == torch.float32 else 2):
        raise ValueError(f"{path}: payload size does not match the shape {shape}")
    if dtype == torch.float32:
        arr = np.frombuffer(payload, dtype="<f4", count=n).astype(np.float32)
        t = torch.from_numpy(arr.copy())
    else:
        arr = np.frombuffer(payload, dtype="<i2", count=n).astype(np.int16)
        t = torch.from_numpy(arr.copy()).view(dtype)
    return t.to(device), layout, header
