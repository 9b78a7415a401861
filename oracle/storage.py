"""Oracle emulation of the stored precision of the rotated slabs.

The estimate-and-prune stage reads the rotated database at a storage
precision; the exact distance is always taken from the original FP32 rows.
The returned arrays hold the stored values exactly, as FP64.

* FP32: round-to-nearest-even of the FP64 rotated value.
* BF16: round-to-nearest-even of the FP32 value to 8 significant bits.
* FP8-E4M3 (the "fn" variant: 4 exponent bits with bias 7, 3 mantissa bits,
  no infinities, largest finite 448, subnormal step 2^-9): per dimension the
  scale is amax_j / 448 over the stored FP32 column (1 if the column is all
  zero); the code is the FP32 quotient x / scale rounded to nearest-even on
  the E4M3 grid and saturated to +-448; the stored value is scale * code.
  The quotient is taken in FP32 because that is the precision in which the
  code is decided.
"""
from __future__ import annotations

import numpy as np


def to_fp32(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def bf16_round(x32: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 round-to-nearest-even, returned as FP32 values."""
    u = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32)


def e4m3_round(y32: np.ndarray) -> np.ndarray:
    """Round FP32 values to the E4M3 grid (nearest, ties to even), saturating
    at +-448.  Returned as FP64 values of the codes."""
    y = np.asarray(y32, dtype=np.float64)
    a = np.abs(y)
    # exponent of the binade; below 2^-6 the grid is the subnormal step 2^-9
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(e, -6.0)
    q = np.exp2(e - 3.0)  # spacing of the grid in this binade
    r = np.round(a / q) * q  # np.round: half to even
    r = np.minimum(r, 448.0)
    return np.sign(y) * r


def fp8_scales(x32: np.ndarray) -> np.ndarray:
    """Per-dimension scale amax_j / 448 as FP32 (1 where the column is zero)."""
    amax = np.abs(np.asarray(x32, dtype=np.float32)).max(axis=0)
    s = (amax / np.float32(448.0)).astype(np.float32)
    s[amax == 0] = np.float32(1.0)
    return s


def stored(xr64: np.ndarray, dtype: str, fp8_scale: np.ndarray | None = None) -> np.ndarray:
    """Stored rotated values, as FP64 arrays, for dtype in {f64, f32, bf16, fp8}
    (f64 keeps the exact rotated values; it exists for the oracle's pins)."""
    if dtype == "f64":
        return np.asarray(xr64, dtype=np.float64)
    x32 = to_fp32(xr64)
    if dtype == "f32":
        return x32.astype(np.float64)
    if dtype == "bf16":
        return bf16_round(x32).astype(np.float64)
    if dtype == "fp8":
        s = fp8_scales(x32) if fp8_scale is None else np.asarray(fp8_scale, dtype=np.float32)
        y = (x32 / s[None, :]).astype(np.float32)
        return e4m3_round(y) * s.astype(np.float64)[None, :]
    raise ValueError(dtype)
