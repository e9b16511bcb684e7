"""Pins of the storage-precision oracle (oracle/precision.py): hand-worked
roundings, the complete e4m3 grid from the format definition, ties, saturation,
the power-of-two tile scale, and agreement with torch's CPU casts (a library
routine) on random data."""
import numpy as np
import pytest

from oracle import precision as P


def test_bf16_hand_values():
    one = 1.0
    cases = [
        (one, one),
        (one + 2.0 ** -8, one),                      # tie between 1 and 1 + 2^-7: even (1) wins
        (one + 3 * 2.0 ** -8, one + 2.0 ** -6),      # tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
        (one + 2.0 ** -8 + 2.0 ** -20, one + 2.0 ** -7),   # just above the tie
        (-(one + 2.0 ** -8 + 2.0 ** -20), -(one + 2.0 ** -7)),
        (3.0, 3.0),
        (0.0, 0.0),
    ]
    got = P.bf16_round(np.array([c[0] for c in cases], dtype=np.float32))
    assert np.array_equal(got, np.array([c[1] for c in cases], dtype=np.float32))


def test_bf16_invariants():
    x = (np.random.default_rng(0).standard_normal(50000) * 10.0 ** np.random.default_rng(1).integers(-20, 20, 50000))
    x = x.astype(np.float32)
    r = P.bf16_round(x)
    assert np.array_equal(P.bf16_round(r), r)                          # idempotent
    assert np.all(r.view(np.uint32) & 0xFFFF == 0)                      # 7 stored mantissa bits
    assert np.all(np.abs(r.astype(np.float64) - x) <= 2.0 ** -8 * np.abs(x.astype(np.float64)))  # half an ulp


def test_bf16_matches_torch_cast():
    torch = pytest.importorskip("torch")
    x = (np.random.default_rng(2).standard_normal(100000) * 37).astype(np.float32)
    ref = torch.tensor(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(P.bf16_round(x), ref)


def _e4m3_grid():
    """All finite non-negative e4m3 values from the format definition:
    exponent field e (4 bits, bias 7), mantissa field f (3 bits); e = 0 is
    subnormal (f/8 * 2^-6); e = 15, f = 7 is NaN."""
    vals = []
    for e in range(16):
        for f in range(8):
            if e == 15 and f == 7:
                continue
            vals.append((f / 8) * 2.0 ** -6 if e == 0 else (1 + f / 8) * 2.0 ** (e - 7))
    return np.array(vals)


def test_e4m3_grid_is_fixed_and_complete():
    g = _e4m3_grid()
    assert len(g) == 127 and g.max() == 448.0 and g[1] == 2.0 ** -9
    assert np.array_equal(P.e4m3_round(g), g)
    assert np.array_equal(P.e4m3_round(-g), -g)


def test_e4m3_ties_go_to_even_mantissa():
    g = _e4m3_grid()
    for i in range(len(g) - 1):
        mid = 0.5 * (g[i] + g[i + 1])
        # index i in the grid has mantissa field i % 8: the even one is chosen
        want = g[i] if i % 2 == 0 else g[i + 1]
        assert P.e4m3_round(mid) == want, (mid, want)
        assert P.e4m3_round(np.nextafter(mid, 0)) == g[i]
        assert P.e4m3_round(np.nextafter(mid, 1e9)) == g[i + 1]


def test_e4m3_saturates():
    assert P.e4m3_round(464.0) == 448.0        # the tie above 448 saturates
    assert P.e4m3_round(1e9) == 448.0
    assert P.e4m3_round(-500.0) == -448.0
    assert P.e4m3_round(2.0 ** -10) == 0.0      # half the smallest subnormal: tie to 0 (even)
    assert P.e4m3_round(3 * 2.0 ** -10) == 2.0 ** -8


def test_e4m3_matches_torch_cast():
    torch = pytest.importorskip("torch")
    x = (np.random.default_rng(3).standard_normal(100000) * 60).astype(np.float32)
    x = np.clip(x, -440, 440)
    ref = torch.tensor(x).to(torch.float8_e4m3fn).double().numpy()
    assert np.array_equal(P.e4m3_round(x.astype(np.float64)), ref)


def test_pow2_tile_scale():
    assert P.pow2_tile_scale(448.0) == 1.0
    assert P.pow2_tile_scale(449.0) == 2.0
    assert P.pow2_tile_scale(224.0) == 0.5
    assert P.pow2_tile_scale(225.0) == 1.0
    assert P.pow2_tile_scale(448.0 * 3) == 4.0
    assert P.pow2_tile_scale(0.0) == 1.0
    assert P.pow2_tile_scale(1e-3) == 2.0 ** -18      # 1e-3 / 448 = 2.23e-6 in (2^-19, 2^-18]


def test_quantize_fp8_tiles():
    rng = np.random.default_rng(4)
    m, n = 300, 260
    A = (rng.standard_normal((m, n)) * np.exp(rng.uniform(-5, 5, (m, 1)))).astype(np.float32)
    A[128:256, 128:256] = 0.0
    vals, sc = P.quantize_fp8(A)
    assert sc.shape == (3, 3) and sc[1, 1] == 1.0 and np.all(vals[128:256, 128:256] == 0)
    for i in range(3):
        for j in range(3):
            blk = A[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128]
            v = vals[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128]
            if np.any(blk):
                # amax / s lies in (224, 448]: the tile's largest code is at least 224
                assert 224.0 <= np.abs(v).max() <= 448.0
                assert np.log2(sc[i, j]) == np.round(np.log2(sc[i, j]))
    deq = P.dequantize_fp8(vals, sc)
    # normal-range values keep 4 significant bits: error at most 2^-4 relative (half an ulp)
    big = np.abs(A) >= 2.0 ** -6 * np.repeat(np.repeat(sc, 128, 0), 128, 1)[:m, :n]
    assert np.all(np.abs(deq - A)[big] <= 2.0 ** -4 * np.abs(A.astype(np.float64))[big])
    assert np.array_equal(P.e4m3_round(vals), vals)
