"""Storage codecs, written from the formats' specifications (test infrastructure only).

The paper stores textures in compressed or reduced formats and decodes one texel per
stochastic lookup (Section 1; Section 5.2, "Texture compression").  The lookup
library keeps dense grids in IEEE binary16 and sparse leaves in OCP FP8 E4M3 with a
per-leaf float32 scale.  Both codecs here are plain definitions:

* binary16: 1 sign bit, 5 exponent bits (bias 15), 10 mantissa bits; subnormals;
  exponent 31 is infinity/NaN.  Encoding is round-to-nearest, ties to the even
  code; magnitudes that round past 65504 become infinity.
* E4M3 (OCP 8-bit floating point, "FN" variant): 1 sign bit, 4 exponent bits
  (bias 7), 3 mantissa bits; subnormals; no infinity; only S.1111.111 is NaN, so
  the largest finite magnitude is 448.  Encoding is round-to-nearest, ties to the
  even code, saturating: finite inputs beyond 448 become +-448.
"""
import numpy as np


def e4m3_decode(code):
    """Exact value of each OCP E4M3 code (bias 7, no infinities, 0x7F/0xFF NaN)."""
    c = np.asarray(code, dtype=np.int64) & 0xFF
    s = np.where(c >> 7, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = (c & 7).astype(np.float64)
    val = np.where(e == 0, m / 8.0 * 2.0 ** -6, (1.0 + m / 8.0) * np.exp2(e - 7.0))
    val = np.where((e == 15) & ((c & 7) == 7), np.nan, val)
    return s * val


def f16_decode(code):
    """Exact value of each IEEE binary16 code."""
    c = np.asarray(code, dtype=np.int64) & 0xFFFF
    s = np.where(c >> 15, -1.0, 1.0)
    e = (c >> 10) & 0x1F
    m = (c & 0x3FF).astype(np.float64)
    val = np.where(e == 0, m / 1024.0 * 2.0 ** -14, (1.0 + m / 1024.0) * np.exp2(e - 15.0))
    val = np.where(e == 31, np.where((c & 0x3FF) == 0, np.inf, np.nan), val)
    return s * val


def _encode_rne(x, pos_codes, pos_values, overflow_code):
    """Nearest representable magnitude, ties to the even code.  ``pos_values`` is
    the increasing table of finite non-negative values with codes ``pos_codes``;
    a magnitude at or beyond the rounding midpoint above the largest value maps to
    ``overflow_code``."""
    x = np.asarray(x, dtype=np.float64)
    sign = np.signbit(x).astype(np.int64)
    a = np.abs(x)
    j = np.clip(np.searchsorted(pos_values, a, side="right") - 1, 0, len(pos_values) - 1)
    lo_v = pos_values[j]
    hi_j = np.minimum(j + 1, len(pos_values) - 1)
    hi_v = pos_values[hi_j]
    d_lo = a - lo_v
    d_hi = hi_v - a
    pick_hi = (d_hi < d_lo) | ((d_hi == d_lo) & (pos_codes[hi_j] % 2 == 0) & (hi_j != j))
    code = np.where(pick_hi, pos_codes[hi_j], pos_codes[j])
    # Beyond the largest finite value: the rounding midpoint to the next (absent)
    # binade step decides overflow.
    top = pos_values[-1]
    step = pos_values[-1] - pos_values[-2]
    code = np.where(a >= top + step / 2, overflow_code, code)
    return code, sign


_E4M3_CODES = np.arange(0, 0x7F, dtype=np.int64)             # +0 .. 448
_E4M3_VALUES = e4m3_decode(_E4M3_CODES)
_F16_CODES = np.arange(0, 0x7C00, dtype=np.int64)             # +0 .. 65504
_F16_VALUES = f16_decode(_F16_CODES)


def e4m3_encode(x):
    """Saturating round-to-nearest-even E4M3 code of each float (NaN -> 0x7F)."""
    x = np.asarray(x, dtype=np.float64)
    code, sign = _encode_rne(x, _E4M3_CODES, _E4M3_VALUES, 0x7E)  # saturate to 448
    code = np.where(np.isinf(x), 0x7E, code)
    code = code | (sign << 7)
    return np.where(np.isnan(x), 0x7F, code).astype(np.uint8)


def f16_encode(x):
    """Round-to-nearest-even binary16 code of each float (overflow -> infinity)."""
    x = np.asarray(x, dtype=np.float64)
    code, sign = _encode_rne(x, _F16_CODES, _F16_VALUES, 0x7C00)
    code = np.where(np.isinf(x), 0x7C00, code)
    code = code | (sign << 15)
    return np.where(np.isnan(x), 0x7E00, code).astype(np.uint16)


def e4m3_leaf_quantise(values32):
    """Per-leaf scaled E4M3 encoding of float32 leaf values, shape (L, 512).

    scale = max|v| / 448 in float32 (1 for an all-zero leaf); code = E4M3(v / scale)
    with the quotient rounded to float32 first, since the decision is taken in the
    float32 precision of the stored values.  Returns (codes uint8 (L, 512),
    scales float32 (L,)).
    """
    v = np.asarray(values32, dtype=np.float32)
    amax = np.max(np.abs(v), axis=1)
    scale = (amax / np.float32(448.0)).astype(np.float32)
    scale = np.where(scale > 0, scale, np.float32(1.0)).astype(np.float32)
    q = (v / scale[:, None]).astype(np.float32)
    return e4m3_encode(q.astype(np.float64)), scale


def e4m3_leaf_dequantise(codes, scales):
    """Exact float64 value of each stored (code, scale) pair."""
    return e4m3_decode(codes) * np.asarray(scales, dtype=np.float64)[..., None]
