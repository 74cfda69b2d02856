"""OCP FP8 E4M3 (the "fn" variant) and the per-block KV quantiser (oracle; test infrastructure only).

E4M3: 1 sign bit, 4 exponent bits with bias 7, 3 mantissa bits; no infinities;
the all-ones pattern S.1111.111 is NaN; the largest finite magnitude is
S.1111.110 = 1.75 * 2^8 = 448; subnormals (exponent field 0) are m * 2^-9.

Quantiser reading (the paper does not use FP8; the precision direction of this
project adds it): the retained KV of one (tuple, layer, kv-head) is cut into
blocks of 64 consecutive slots in retention rank order, K and V separately;
``scale = amax / 448`` over the block (``scale = 1`` when amax = 0);
``code = RN-even(x / scale)`` saturated to +-448; the dequantised value is
``decode(code) * scale``.
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0
BLOCK = 64


def e4m3_decode(code: int) -> float:
    """Value of one E4M3 byte from its bit fields."""
    code = int(code) & 0xFF
    sign = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 0x7
    if e == 0xF and m == 0x7:
        return float("nan")
    if e == 0:
        return sign * m * 2.0 ** -9
    return sign * (1.0 + m / 8.0) * 2.0 ** (e - 7)


# Non-negative finite grid, codes 0x00 .. 0x7E, increasing with the code.
_GRID = np.array([e4m3_decode(c) for c in range(0x7F)], dtype=np.float64)


def e4m3_encode(x) -> np.ndarray:
    """Round each value to the nearest E4M3 code, ties to the even code, saturating to +-448.

    Input may be float32 or float64; the decision is taken on the given value
    exactly (no intermediate rounding).  NaN maps to 0x7F.
    """
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), E4M3_MAX)
    hi = np.searchsorted(_GRID, a, side="left").clip(0, len(_GRID) - 1)   # first grid >= a
    lo = np.maximum(hi - 1, 0)
    d_lo = a - _GRID[lo]
    d_hi = _GRID[hi] - a
    pick_hi = (d_hi < d_lo) | ((d_hi == d_lo) & (hi % 2 == 0))
    code = np.where(pick_hi, hi, lo).astype(np.uint8)
    neg = np.signbit(x)
    code = np.where(neg, code | 0x80, code).astype(np.uint8)
    return np.where(np.isnan(x), np.uint8(0x7F), code).astype(np.uint8)


def e4m3_decode_array(codes) -> np.ndarray:
    codes = np.asarray(codes, dtype=np.uint8)
    mag = _GRID[np.minimum(codes & 0x7F, 0x7E)]
    out = np.where(codes & 0x80, -mag, mag)
    return np.where((codes & 0x7F) == 0x7F, np.nan, out)


def quantize_blocks(x: np.ndarray, arith: str = "f64"):
    """Quantise ``x[n, hd]`` (rank-ordered slots of one tuple, layer and kv head).

    Returns ``(codes uint8[n, hd], scales[ceil(n/64)], dequant float64[n, hd])``.
    ``arith = "f32"`` takes the scale and the division in IEEE float32 (the
    precision in which the CUDA kernel decides the codes); ``"f64"`` in float64.
    """
    x = np.asarray(x)
    n = x.shape[0]
    nb = (n + BLOCK - 1) // BLOCK
    codes = np.zeros(x.shape, dtype=np.uint8)
    deq = np.zeros(x.shape, dtype=np.float64)
    scales = np.zeros(nb, dtype=np.float64 if arith == "f64" else np.float32)
    for b in range(nb):
        blk = x[b * BLOCK:(b + 1) * BLOCK]
        if arith == "f32":
            blk = blk.astype(np.float32)
            amax = np.float32(np.max(np.abs(blk))) if blk.size else np.float32(0)
            scale = np.float32(1.0) if amax == 0 else np.float32(amax / np.float32(E4M3_MAX))
            y = (blk / scale).astype(np.float32)
        else:
            blk = blk.astype(np.float64)
            amax = np.max(np.abs(blk)) if blk.size else 0.0
            scale = 1.0 if amax == 0 else amax / E4M3_MAX
            y = blk / scale
        c = e4m3_encode(y)
        codes[b * BLOCK:(b + 1) * BLOCK] = c
        deq[b * BLOCK:(b + 1) * BLOCK] = e4m3_decode_array(c) * np.float64(scale)
        scales[b] = scale
    return codes, scales, deq
