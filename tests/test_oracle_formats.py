"""Pins for the oracle's number formats (not GPU).

bfloat16 rounding and OCP FP8 E4M3 encoding/decoding are pinned against
PyTorch's CPU conversions (library routines) over every rounding boundary;
the FP8 saturation rule ("satfinite": finite overflow clamps to +-448) and the
per-row scale are pinned by their definitions.
"""
import numpy as np
import pytest
import torch

import oracle
from tests import inputs


def _bf16_torch(f32: np.ndarray) -> np.ndarray:
    t = torch.from_numpy(f32.astype(np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16)


def test_bf16_matches_torch_on_all_rounding_boundaries():
    hi = np.arange(0, 1 << 16, 7, dtype=np.uint64)
    lows = np.array([0x0000, 0x0001, 0x7FFF, 0x8000, 0x8001, 0xFFFF], dtype=np.uint64)
    bits = ((hi[:, None] << 16) | lows[None, :]).ravel().astype(np.uint32)
    f = bits.view(np.float32)
    finite = np.isfinite(f)
    want = _bf16_torch(f[finite])
    got = np.array([oracle.bf16_rne(float(v)) for v in f[finite]], dtype=np.uint16)
    assert np.array_equal(got, want)


def test_bf16_random_values():
    f = inputs.rng(5).standard_normal(20000).astype(np.float32) * np.float32(0.3)
    want = _bf16_torch(f)
    got = np.array([oracle.bf16_rne(float(v)) for v in f], dtype=np.uint16)
    assert np.array_equal(got, want)
    back = np.array([oracle.bf16_value(int(b)) for b in got])
    ref = torch.from_numpy(want.view(np.int16)).view(torch.bfloat16).float().numpy()
    assert np.array_equal(back, ref.astype(np.float64))


def test_e4m3_decode_all_codes_matches_torch():
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    got = np.array([oracle.e4m3_value(int(c)) for c in codes])
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan], ref[~nan])
    assert oracle.e4m3_value(0x7E) == 448.0 and oracle.e4m3_value(0x01) == 2.0**-9


def test_e4m3_encode_matches_torch_at_every_midpoint():
    vals = np.array(sorted({oracle.e4m3_value(c) for c in range(0, 0x7F)}), dtype=np.float64)
    mids = (vals[:-1] + vals[1:]) / 2  # exact ties (binary32-representable here)
    probe = []
    for m in mids:
        m32 = np.float32(m)
        assert float(m32) == m
        probe += [m32, np.nextafter(m32, np.float32(0)), np.nextafter(m32, np.float32(1e9))]
    probe += list(vals.astype(np.float32))
    probe = np.array(probe, dtype=np.float32)
    probe = np.concatenate([probe, -probe])
    probe = probe[np.abs(probe) < 464.0]  # torch maps >= 464 to NaN; we saturate
    want = torch.from_numpy(probe).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = np.array([oracle.e4m3_encode(float(v)) for v in probe], dtype=np.uint8)
    assert np.array_equal(got, want)


def test_e4m3_encode_random_values_match_torch():
    f = (inputs.rng(6).standard_normal(20000) * 60).astype(np.float32)
    f = f[np.abs(f) < 464.0]
    want = torch.from_numpy(f).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = np.array([oracle.e4m3_encode(float(v)) for v in f], dtype=np.uint8)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("v", [448.0, 449.0, 463.9, 464.0, 480.0, 1e6, 3e38, float("inf")])
def test_e4m3_satfinite_clamps(v):
    assert oracle.e4m3_encode(v) == 0x7E
    assert oracle.e4m3_encode(-v) == 0xFE


def test_fp8_row_scale_definition():
    rows = inputs.random_params(371, n_rows=50, seed=7)
    for row in rows:
        want = np.float32(np.max(np.abs(row))) / np.float32(448.0)  # IEEE binary32 division
        assert oracle.fp8_row_scale(row) == float(want)
    assert oracle.fp8_row_scale(np.zeros(64, np.float32)) == 1.0
