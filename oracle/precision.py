"""Storage precisions of A for the low-precision passes (test infrastructure only).

Plain numpy definitions of the two storage conversions the GPU library offers
for A, used by the tests to check its quantiser bit for bit and to build the
dequantised matrix the FP64 oracle runs on.  The paper fixes no storage
precision (it works in double precision throughout); these conversions are the
library's own, written here from the IEEE / OCP format definitions:

  bf16_round        FP32 -> bfloat16 (8 exponent bits, 7 stored mantissa bits),
                    round to nearest, ties to even
  e4m3_round        real -> FP8 e4m3 value (bias 7, 3 stored mantissa bits,
                    largest finite 448, subnormal step 2^-9, no infinities),
                    round to nearest, ties to even, saturating at +-448
  pow2_tile_scale   smallest power of two >= fl32(amax / 448)
  quantize_fp8      per-128 x 128-tile scales and e4m3 values of A / scale
  dequantize_fp8    e4m3 value x tile scale (exact in float64)

Imported only by tests/; shares no code with the CUDA path.
Pins: tests/test_oracle_precision.py (hand-worked values, the format's
grid and extremes, ties, agreement with torch's CPU casts, invariants).
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0
TILE = 128


def bf16_round(x) -> np.ndarray:
    """FP32 values rounded to bfloat16 (nearest, ties to even), returned as float32.

    A bfloat16 is the upper 16 bits of an FP32: rounding adds half of the
    dropped range minus one, plus the lowest kept bit (ties go to even), then
    clears the low 16 bits.  Finite inputs only."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    keep_lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = (b + np.uint64(0x7FFF) + keep_lsb) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32)


def e4m3_round(x) -> np.ndarray:
    """Real values rounded to the e4m3 grid (nearest, ties to even, saturating), float64.

    Normal binades [2^e, 2^(e+1)) for e = -6 .. 8 hold 8 values spaced 2^(e-3);
    below 2^-6 the subnormals are spaced 2^-9.  The quotient |x| / spacing is
    rounded half-to-even, which is ties-to-even on the last mantissa bit."""
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    _, E = np.frexp(ax)                 # ax = f 2^E, f in [0.5, 1): binade exponent E - 1
    e = np.maximum(E - 1, -6)
    step = np.ldexp(1.0, e - 3)
    r = np.round(ax / step) * step      # numpy rounds halves to even
    r = np.minimum(r, E4M3_MAX)
    return np.copysign(r, x)


def pow2_tile_scale(amax: float) -> float:
    """Smallest power of two >= fl32(amax / 448); 1 for an all-zero tile.

    The quotient is taken in FP32, the precision the GPU quantiser uses to
    decide the exponent."""
    if amax == 0.0:
        return 1.0
    x = np.float32(amax) / np.float32(E4M3_MAX)
    f, E = np.frexp(np.float64(x))     # x = f 2^E exactly
    if x < np.float32(2.0 ** -126):
        return 2.0 ** -126
    return float(np.ldexp(1.0, int(E) - 1)) if f == 0.5 else float(np.ldexp(1.0, int(E)))


def quantize_fp8(A32) -> tuple[np.ndarray, np.ndarray]:
    """Per-128 x 128-tile FP8 e4m3 storage of an FP32 matrix.

    Returns (values, scales): values[i, j] is the e4m3 value of
    A[i, j] / scale[i // 128, j // 128] (float64), scales the power-of-two tile
    scales (float64, ceil(m/128) x ceil(n/128))."""
    A = np.asarray(A32, dtype=np.float32)
    m, n = A.shape
    tr, tc = -(-m // TILE), -(-n // TILE)
    scales = np.empty((tr, tc), dtype=np.float64)
    vals = np.empty((m, n), dtype=np.float64)
    for i in range(tr):
        for j in range(tc):
            blk = A[i * TILE:(i + 1) * TILE, j * TILE:(j + 1) * TILE].astype(np.float64)
            s = pow2_tile_scale(float(np.max(np.abs(blk))) if blk.size else 0.0)
            scales[i, j] = s
            vals[i * TILE:(i + 1) * TILE, j * TILE:(j + 1) * TILE] = e4m3_round(blk / s)
    return vals, scales


def dequantize_fp8(vals, scales) -> np.ndarray:
    """e4m3 values times their tile scales (float64, exact for power-of-two scales)."""
    vals = np.asarray(vals, dtype=np.float64)
    s = np.repeat(np.repeat(np.asarray(scales, dtype=np.float64), TILE, axis=0), TILE, axis=1)
    return vals * s[:vals.shape[0], :vals.shape[1]]
