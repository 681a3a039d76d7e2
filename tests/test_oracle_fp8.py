"""Pins for the oracle's E4M3 encoder/decoder and quantiser (CPU only).

Pinned against the OCP OFP8 definition's named values and against torch's
float8_e4m3fn conversions (an independent library routine), plus
round-trip and tie-breaking cases chosen by hand.
"""
import numpy as np
import pytest
import torch

from oracle import fp8
import workloads


def test_named_values():
    d = fp8.decode_e4m3
    assert d(0x7E) == 448.0                  # S.1111.110 max finite
    assert d(0xFE) == -448.0
    assert d(0x01) == 2.0 ** -9              # smallest subnormal
    assert d(0x07) == 7 * 2.0 ** -9          # largest subnormal
    assert d(0x08) == 2.0 ** -6              # smallest normal
    assert d(0x38) == 1.0
    assert d(0xC0) == -2.0
    assert d(0x00) == 0.0 and np.signbit(d(0x80))
    assert np.isnan(d(0x7F)) and np.isnan(d(0xFF))


def test_decode_matches_torch_all_codes():
    codes = np.arange(256, dtype=np.uint8)
    ours = fp8.decode_e4m3(codes)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])


def test_round_trip():
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF)], dtype=np.uint8)
    assert np.array_equal(fp8.encode_e4m3(fp8.decode_e4m3(codes)), codes)


def test_ties_to_even_and_saturation():
    e = fp8.encode_e4m3
    assert e(1.0625) == 0x38      # halfway 1.0 (m=0) / 1.125 (m=1) -> even
    assert e(1.1875) == 0x3A      # halfway 1.125 (m=1) / 1.25 (m=2) -> even
    assert e(-1.0625) == 0xB8
    assert e(2.0 ** -10) == 0x00  # halfway 0 / smallest subnormal -> 0
    assert e(3 * 2.0 ** -10) == 0x02   # halfway m=1 / m=2 -> m=2
    assert e(1000.0) == 0x7E and e(-1e9) == 0xFE and e(464.0) == 0x7E
    assert e(np.nan) == 0x7F


def test_encode_matches_torch_in_range():
    x = workloads.normal((20000,), seed=21).numpy() * 60.0
    x = np.clip(x, -448.0, 448.0).astype(np.float32)
    ours = fp8.encode_e4m3(x)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, ref)


def test_quantize_scale_and_extremes():
    x = workloads.normal((64, 80), seed=22).numpy()
    codes, s = fp8.quantize_e4m3(x)
    amax = np.float32(np.max(np.abs(x)))
    assert s == np.float32(amax / np.float32(448.0))
    deq = fp8.dequantize_e4m3(codes, s)
    # the largest-magnitude element maps to +-448 (or the code just below it
    # when float32(amax / s) rounds under 448)
    k = np.argmax(np.abs(x))
    assert abs(fp8.decode_e4m3(codes.flat[k])) >= 416.0
    # every value within half an E4M3 ulp (relative 2^-4) of x, or of the
    # subnormal spacing near zero
    err = np.abs(deq - x.astype(np.float64))
    assert np.all(err <= np.maximum(2.0 ** -4 * np.abs(x), 2.0 ** -10 * s) + 1e-30)
    z_codes, z_s = fp8.quantize_e4m3(np.zeros(5, np.float32))
    assert z_s == 1.0 and np.all(z_codes == 0)
