"""FP8 E4M3 encode/decode and per-tensor quantisation -- TEST INFRASTRUCTURE ONLY.

Written from the OCP 8-bit floating point (OFP8) definition of E4M3:
1 sign bit, 4 exponent bits with bias 7, 3 mantissa bits, no infinities,
the single NaN pattern S.1111.111, largest finite magnitude
S.1111.110 = 1.75 * 2^8 = 448.  Exponent field 0 encodes subnormals
m/8 * 2^-6.

Encoding here is by brute force over the 127 non-negative finite codes:
round to the nearest representable value, ties to the code with an even
mantissa, and saturate magnitudes above 448 to 448 (the "satfinite"
conversion).

Quantisation reading (the paper gives none; this is the per-tensor scaled
form of the FP8 workload): scale = amax / 448 in float32, amax = max |x|;
scale = 1 if amax == 0; q = E4M3(float32(x / scale)).  The division is a
float32 division, the same precision the GPU kernel uses, because it decides
an integer code.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0
E4M3_NAN = 0x7F


def decode_e4m3(code) -> np.ndarray:
    """Decode uint8 E4M3 codes to float64 values (NaN for 0x7F / 0xFF)."""
    c = np.asarray(code, dtype=np.uint8).astype(np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = c & 0x7
    sub = (m / 8.0) * 2.0 ** -6
    norm = (1.0 + m / 8.0) * np.power(2.0, (e - 7).astype(np.float64))
    val = np.where(e == 0, sub, norm) * sign
    nan = (e == 0xF) & (m == 0x7)
    return np.where(nan, np.nan, val)


# Non-negative finite codes 0x00..0x7E in increasing order of value.
_POS_CODES = np.arange(0x7F, dtype=np.uint8)
_POS_VALS = decode_e4m3(_POS_CODES)
assert np.all(np.diff(_POS_VALS) > 0)


def encode_e4m3(x) -> np.ndarray:
    """Round float values to E4M3 codes: nearest, ties to even mantissa,
    saturating to +-448; NaN maps to 0x7F."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    a_sat = np.minimum(a, E4M3_MAX)
    hi = np.searchsorted(_POS_VALS, a_sat, side="left")
    hi = np.clip(hi, 0, len(_POS_VALS) - 1)
    lo = np.clip(hi - 1, 0, len(_POS_VALS) - 1)
    d_hi = _POS_VALS[hi] - a_sat
    d_lo = a_sat - _POS_VALS[lo]
    pick_lo = (d_lo < d_hi) | ((d_lo == d_hi) & ((_POS_CODES[lo] & 1) == 0))
    idx = np.where(pick_lo, lo, hi)
    code = _POS_CODES[idx].astype(np.uint8)
    # The sign bit is copied, so negative values that round to zero give
    # the negative-zero code 0x80, as an IEEE-style conversion does.
    code = np.where(np.signbit(x), code | np.uint8(0x80), code)
    code = np.where(np.isnan(x), np.uint8(E4M3_NAN), code)
    return code.astype(np.uint8)


def quant_scale(x) -> np.float32:
    """Per-tensor scale amax / 448 in float32 (1 when the tensor is all zero)."""
    x32 = np.asarray(x, dtype=np.float32)
    amax = np.float32(np.max(np.abs(x32))) if x32.size else np.float32(0)
    if amax == 0:
        return np.float32(1.0)
    return np.float32(amax / np.float32(E4M3_MAX))


def quantize_e4m3(x):
    """Return (codes uint8, scale float32) for a float32 tensor."""
    x32 = np.asarray(x, dtype=np.float32)
    s = quant_scale(x32)
    q = (x32 / s).astype(np.float32)
    return encode_e4m3(q), s


def dequantize_e4m3(codes, scale) -> np.ndarray:
    """Exact float64 values code * scale."""
    return decode_e4m3(codes) * np.float64(scale)
