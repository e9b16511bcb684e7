"""Counter-based random numbers shared by every harness (test inputs only).

Every value is addressed by (seed, index), so any element, slice or whole
matrix can be regenerated on its own, on the CPU (numpy) or on a device
(torch), without drawing the elements before it.

Definition (SplitMix64, Steele, Lea & Flood, OOPSLA 2014; the reference
stream of S. Vigna's splitmix64.c):

    h(seed, i) = mix(seed + (i + 1) * 0x9E3779B97F4A7C15   mod 2^64)
    mix(z):  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
             z = (z ^ (z >> 27)) * 0x94D049BB133111EB
             z =  z ^ (z >> 31)

i.e. h(seed, i) is output number i of a SplitMix64 generator whose state
starts at `seed`.  From it:

    uniform01(seed, i) = (h(seed, i) >> 11) * 2^-53            in [0, 1)
    normal(seed, e)    = sqrt(-2 ln u1) * cos(2 pi u2)          (Box-Muller)
        u1 = ((h(seed, 2e) >> 11) + 1) * 2^-53                 in (0, 1]
        u2 =  (h(seed, 2e + 1) >> 11) * 2^-53

The integer part is bit-identical on both backends; the Box-Muller
transcendental functions are evaluated in float64 by each backend's own
libm, which may differ in the last unit of the float64 result.  Parity
tests therefore generate on the CPU and copy the very same array to the GPU.

This module holds no arithmetic of the factorisation method.
"""
from __future__ import annotations

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
_TWO53 = float(2 ** -53)


def stream_seed(base: int, sub: int = 0) -> int:
    """Seed of sub-stream `sub` of a base seed (distinct matrices of one input)."""
    return (base * 1000003 + sub * 7919 + 1) & ((1 << 64) - 1)


# --------------------------------------------------------------------------- numpy
def _mix_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
    return z ^ (z >> np.uint64(31))


def hash_np(seed: int, idx: np.ndarray) -> np.ndarray:
    """h(seed, idx) for a uint64 index array."""
    with np.errstate(over="ignore"):
        idx = idx.astype(np.uint64, copy=False)
        z = np.uint64(seed & ((1 << 64) - 1)) + (idx + np.uint64(1)) * np.uint64(GOLDEN)
        return _mix_np(z)


def uniform_np(seed: int, idx: np.ndarray) -> np.ndarray:
    return (hash_np(seed, idx) >> np.uint64(11)).astype(np.float64) * _TWO53


def normal_np(seed: int, idx: np.ndarray) -> np.ndarray:
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h1 = hash_np(seed, idx * np.uint64(2))
        h2 = hash_np(seed, idx * np.uint64(2) + np.uint64(1))
    u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) * _TWO53
    u2 = (h2 >> np.uint64(11)).astype(np.float64) * _TWO53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def normal_block_np(seed: int, n_cols_total: int, r0: int, r1: int, c0: int, c1: int) -> np.ndarray:
    """Rows r0:r1, columns c0:c1 of the logical row-major matrix with
    n_cols_total columns whose element (r, c) is normal(seed, r*n_cols_total + c)."""
    r = np.arange(r0, r1, dtype=np.uint64)[:, None]
    c = np.arange(c0, c1, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        idx = r * np.uint64(n_cols_total) + c
    return normal_np(seed, idx)


def uniform_block_np(seed: int, n_cols_total: int, r0: int, r1: int, c0: int, c1: int) -> np.ndarray:
    r = np.arange(r0, r1, dtype=np.uint64)[:, None]
    c = np.arange(c0, c1, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        idx = r * np.uint64(n_cols_total) + c
    return uniform_np(seed, idx)


# --------------------------------------------------------------------------- torch
def _as_i64(v: int) -> int:
    v &= (1 << 64) - 1
    return v - (1 << 64) if v >= (1 << 63) else v


def _lsr(z, s: int):
    """Logical right shift of an int64 tensor holding uint64 bit patterns."""
    import torch
    return torch.bitwise_and(torch.bitwise_right_shift(z, s), (1 << (64 - s)) - 1)


def _mix_t(z):
    z = torch_mul_wrap(torch_xor(z, _lsr(z, 30)), _as_i64(MIX1))
    z = torch_mul_wrap(torch_xor(z, _lsr(z, 27)), _as_i64(MIX2))
    return torch_xor(z, _lsr(z, 31))


def torch_xor(a, b):
    import torch
    return torch.bitwise_xor(a, b)


def torch_mul_wrap(a, c: int):
    """a * c modulo 2^64 on int64 tensors (two's complement wrap-around).

    Split into 32-bit halves so that no signed product overflows:
    (ah*2^32 + al) * (ch*2^32 + cl) = al*cl + ((ah*cl + al*ch) << 32)  mod 2^64.
    """
    import torch
    mask32 = 0xFFFFFFFF
    al = torch.bitwise_and(a, mask32)
    ah = torch.bitwise_and(_lsr(a, 32), mask32)
    cu = c & ((1 << 64) - 1)
    cl = cu & mask32
    ch = (cu >> 32) & mask32
    # the product of two values < 2^32 can exceed 2^63: _mul32x32_wrap splits it
    low = _mul32x32_wrap(al, cl)
    cross = torch.bitwise_and(_mul32x32_wrap(ah, cl) + _mul32x32_wrap(al, ch), mask32)
    return low + torch.bitwise_left_shift(cross, 32)


def _mul32x32_wrap(x, c: int):
    """x * c mod 2^64 for 0 <= x, c < 2^32 without signed overflow."""
    import torch
    c_lo = c & 0xFFFF
    c_hi = c >> 16
    # x * c = x*c_lo + (x*c_hi << 16); x*c_lo < 2^48, x*c_hi < 2^48
    return x * c_lo + torch.bitwise_left_shift(x * c_hi, 16)


def hash_t(seed: int, idx):
    """h(seed, idx) for an int64 index tensor (any device)."""
    z = torch_mul_wrap(idx + 1, _as_i64(GOLDEN)) + _as_i64(seed)
    return _mix_t(z)


def normal_t(seed: int, idx):
    import torch
    h1 = hash_t(seed, idx * 2)
    h2 = hash_t(seed, idx * 2 + 1)
    u1 = (_lsr(h1, 11).to(torch.float64) + 1.0) * _TWO53
    u2 = _lsr(h2, 11).to(torch.float64) * _TWO53
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * np.pi * u2)


def uniform_t(seed: int, idx):
    import torch
    return _lsr(hash_t(seed, idx), 11).to(torch.float64) * _TWO53


def normal_block_t(seed: int, n_cols_total: int, r0: int, r1: int, c0: int, c1: int,
                   device="cpu", chunk_rows: int | None = None):
    """Torch twin of normal_block_np (float64), generated on `device`."""
    import torch
    rows = r1 - r0
    cols = c1 - c0
    out = torch.empty((rows, cols), dtype=torch.float64, device=device)
    if chunk_rows is None:
        chunk_rows = max(1, (1 << 24) // max(cols, 1))
    c = torch.arange(c0, c1, dtype=torch.int64, device=device)[None, :]
    for a in range(0, rows, chunk_rows):
        b = min(rows, a + chunk_rows)
        r = torch.arange(r0 + a, r0 + b, dtype=torch.int64, device=device)[:, None]
        out[a:b] = normal_t(seed, r * n_cols_total + c)
    return out


def uniform_block_t(seed: int, n_cols_total: int, r0: int, r1: int, c0: int, c1: int,
                    device="cpu", chunk_rows: int | None = None):
    import torch
    rows = r1 - r0
    cols = c1 - c0
    out = torch.empty((rows, cols), dtype=torch.float64, device=device)
    if chunk_rows is None:
        chunk_rows = max(1, (1 << 24) // max(cols, 1))
    c = torch.arange(c0, c1, dtype=torch.int64, device=device)[None, :]
    for a in range(0, rows, chunk_rows):
        b = min(rows, a + chunk_rows)
        r = torch.arange(r0 + a, r0 + b, dtype=torch.int64, device=device)[:, None]
        out[a:b] = uniform_t(seed, r * n_cols_total + c)
    return out
