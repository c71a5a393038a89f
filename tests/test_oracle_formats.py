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


def _logical_rows(D, H, A, L, ns):
    """Weight rows of the logical parameter order (W_in [H][D], ns input
    biases [H], L x (W_l [H][H], b_l [H]), W_out [A][H], then the head bias
    or the temperature): (start, length) of every weight row, in the order
    W_in, hidden layers, head."""
    rows = [(o * D, D) for o in range(H)]
    hid0 = H * D + ns * H
    for l in range(L):
        rows += [(hid0 + l * (H * H + H) + o * H, H) for o in range(H)]
    out0 = hid0 + L * (H * H + H)
    rows += [(out0 + a * H, H) for a in range(A)]
    return rows


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("form,over", [
    ("plain", dict()),
    ("plain", dict(patch_k=5, n_scalars=4, hidden=32, n_actions=6)),
    ("paper", dict(n_hidden=1, hidden=32)),
    ("paper", dict(n_hidden=3, hidden=128)),
    ("paper", dict(n_hidden=2, patch_k=0)),           # blind: D below H
])
def test_quantise_matches_torch_row_by_row(prec, form, over):
    """The oracle's streamed copy of whole master rows (codes in logical
    order, FP8 row scales) against torch's bfloat16 / float8_e4m3fn
    conversions applied row by row to the weights, with numpy's binary32
    max / 448 as the row scale; biases and the temperature keep the code 0."""
    from paper_2510_18221_gb300 import workloads
    w = workloads.get("mid", precision=prec, policy_form=form, side=16, slots=4, init_alive=0,
                      **over)
    orc = oracle.Oracle(w)
    D, H, A = orc.D, w["hidden"], w["n_actions"]
    L = w.get("n_hidden", 1) if form == "paper" else 1
    ns = 1 if form == "plain" else (1 if w["patch_k"] > 0 else 0) + (1 if w["n_scalars"] >= 8 else 0) + 1
    rows = _logical_rows(D, H, A, L, ns)
    n_w = sum(n for _, n in rows)
    wmask = np.zeros(orc.P, bool)
    for s, n in rows:
        wmask[s:s + n] = True
    assert n_w == H * D + L * H * H + A * H
    assert np.array_equal(orc.weight_mask(), wmask)
    m = inputs.random_params(orc.P, n_rows=5, seed=11)
    m[1] = 0.0                                   # all-zero rows: scale 1
    m[2, :n_w // 3] *= np.float32(1e-4)          # e4m3 subnormal codes
    m[3] *= np.float32(50.0)                     # large magnitudes
    codes, scales = orc.quantise(m)
    assert not codes[:, ~wmask].any()
    for i in range(m.shape[0]):
        if prec == "bf16":
            assert np.array_equal(codes[i, wmask], _bf16_torch(m[i, wmask]))
            continue
        assert scales.shape[1] == len(rows)
        for r, (s, n) in enumerate(rows):
            row = m[i, s:s + n]
            mx = np.float32(np.max(np.abs(row)))
            want_s = np.float32(1.0) if mx == 0 else mx / np.float32(448.0)
            assert scales[i, r] == want_s, (i, r)
            q = (row / want_s).astype(np.float32)     # binary32 division
            want = torch.from_numpy(q).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
            assert np.array_equal(codes[i, s:s + n], want), (i, r)
