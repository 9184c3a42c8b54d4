"""PSF bank files: round trip of every storage type and field mode, and the
checks that refuse a damaged file or a bank traced with another lens."""
import numpy as np
import pytest
import torch

import paper_2503_11213_gb300 as sd
import workloads as W


def make(dtype, mode, nl=3, ks=9):
    fh = np.array([0.0, 0.3, 0.7], dtype=np.float32)
    dm = np.array([0.5, 1.0, 2.5, 4.0], dtype=np.float32)
    lay = sd.BankLayout(fh, dm, nl, ks, 0.004, dtype=dtype, field_mode=mode)
    g = torch.Generator().manual_seed(5)
    bank = torch.rand(int(np.prod(lay.shape())), generator=g).to(dtype)
    return bank, lay


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("mode", [sd.SD_FIELD_RADIAL, sd.SD_FIELD_QUADRANT])
def test_round_trip(tmp_path, dtype, mode):
    bank, lay = make(dtype, mode)
    lens = W.doublet_pair_f18()
    sensor = sd.DPSensor(0.004)
    p = tmp_path / "bank.sdb"
    sd.save_bank(p, bank, lay, lens_table=lens, sensor=sensor, lambdas_nm=[460.0, 550.0, 640.0])
    got, lay2, hdr = sd.load_bank(p, device="cpu", lens_table=lens)
    assert got.dtype == dtype and got.shape == bank.shape
    assert torch.equal(got.view(torch.int16) if dtype != torch.float32 else got,
                       bank.view(torch.int16) if dtype != torch.float32 else bank)
    assert lay2.shape() == lay.shape() and lay2.dtype == lay.dtype
    assert lay2.field_mode == mode and lay2.ks == lay.ks and lay2.n_lambda == lay.n_lambda
    np.testing.assert_array_equal(lay2.fh, lay.fh)
    np.testing.assert_array_equal(lay2.dm, lay.dm)
    assert abs(lay2.pitch_mm - lay.pitch_mm) == 0.0
    assert hdr["sensor"]["pitch_mm"] == 0.004 and hdr["lambdas_nm"] == [460.0, 550.0, 640.0]
    assert hdr["lens_sha256"] == sd.lens_sha256(lens)


def test_rejects_wrong_lens_and_damage(tmp_path):
    bank, lay = make(torch.float32, sd.SD_FIELD_RADIAL)
    p = tmp_path / "bank.sdb"
    sd.save_bank(p, bank, lay, lens_table=W.doublet_pair_f18())
    with pytest.raises(ValueError, match="another lens"):
        sd.load_bank(p, device="cpu", lens_table=W.singlet_f2())
    data = bytearray(p.read_bytes())
    data[-5] ^= 0x40                                       # one flipped payload bit
    q = tmp_path / "flipped.sdb"
    q.write_bytes(bytes(data))
    with pytest.raises(ValueError, match="checksum"):
        sd.load_bank(q, device="cpu")
    q.write_bytes(p.read_bytes()[:-8])                     # truncated payload
    with pytest.raises(ValueError, match="payload"):
        sd.load_bank(q, device="cpu")
    q.write_bytes(b"NOTABANK" + p.read_bytes()[8:])
    with pytest.raises(ValueError, match="not a PSF bank"):
        sd.load_bank(q, device="cpu")
    d = bytearray(p.read_bytes())
    d[6] = 9                                               # a future format version
    q.write_bytes(bytes(d))
    with pytest.raises(ValueError, match="version"):
        sd.load_bank(q, device="cpu")


def test_save_checks_the_bank_against_the_layout(tmp_path):
    bank, lay = make(torch.float32, sd.SD_FIELD_RADIAL)
    with pytest.raises(ValueError, match="dtype"):
        sd.save_bank(tmp_path / "a.sdb", bank.to(torch.bfloat16), lay)
    with pytest.raises(ValueError, match="elements"):
        sd.save_bank(tmp_path / "b.sdb", bank[:-1], lay)


def test_traced_bank_layout_matches_the_request_order():
    # the bank a bank_grid request array traces is [field][depth][lambda][2][ks][ks],
    # i.e. layout.shape() for a radial layout of the same grid
    c = W.config_singlet()
    reqs = W.bank_grid(c["field_h_mm"], c["depths_mm"], c["lambdas_nm"], c["n_grid"], c["ks"])
    lay = sd.BankLayout(c["field_h_mm"], c["depths_mm"] / 1000.0, len(c["lambdas_nm"]), c["ks"],
                        c["pitch_mm"])
    assert int(np.prod(lay.shape())) == int((2 * reqs["ks"].astype(np.int64) ** 2).sum())
