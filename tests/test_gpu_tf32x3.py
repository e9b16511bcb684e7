"""GPU parity of the split-operand pass (mma "tf32x3", the FP32-class tensor-core
engine) through the C ABI, against the FP64 product of the same FP32 inputs.

Bound.  Each FP32 value v is split as v = h + c + r with h = TF32(v) and
c = BF16(v - h), both to nearest (unit roundoffs 2^-11 and 2^-8), so
|v - h| <= 2^-11 |v| and |r| <= 2^-8 |v - h| <= 2^-19 |v|.  The pass forms
h_a h_x exactly (a TF32 x TF32 product fits FP32) plus the BF16 MMA
c_a bf16(h_x) + bf16(h_a) c_x, whose two terms are each within 2^-8 of
c_a h_x and h_a c_x (<= 2^-19 |a x|).  What the product misses is r_a x + a r_x
(<= 2^-18 |a x|), the two BF16 roundings (<= 2^-18) and c_a c_x (<= 2^-22): at
most 2^-16.9 |a x|.  The tensor core accumulates the 2K/8 MMA results in FP32
(at most one unit of 2^-23 of the running sum per addition, allowing for
truncation).  Hence
    |C - C_ref| <= (2^-16.9 + (2K + 8) 2^-23) (|X| |A|)            (deterministic)
The rounding errors are zero-mean and independent, so against the natural scale
s = sqrt((X o X)(A o A)) they stay near 2^-18; the test asks
max |C - C_ref| / s <= 2^-14, which a pass that dropped either cross term
(errors ~2^-12 s) fails.
"""
import numpy as np
import pytest

from oracle import corutv_oracle as O
from synth import counter as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1810_07323_gb300 import corutv


def _gauss(seed, r, c):
    return C.normal_block_np(seed, c, 0, r, 0, c)


def _st(host, ld_len):
    l, n = host.shape
    buf = torch.zeros((l, corutv.ld_for(ld_len)), dtype=torch.float32, device="cuda")
    buf[:, :n] = torch.tensor(host, dtype=torch.float32, device="cuda")
    return buf


def _dev(A):
    m, n = A.shape
    lda = -(-n // 4) * 4 + 4          # 16-byte row pitch, lda > n
    buf = torch.zeros((m, lda), dtype=torch.float32, device="cuda")[:, :n]
    buf.copy_(torch.tensor(A, dtype=torch.float32, device="cuda"))
    return buf


def _check(got, ref, X, Aop, K):
    err = np.abs(got - ref)
    det = (2.0 ** -16.9 + (2 * K + 8) * 2.0 ** -23) * (np.abs(X) @ np.abs(Aop))
    assert np.all(err <= det + 1e-30), float(np.max(err / (det + 1e-300)))
    s = np.sqrt((X * X) @ (Aop * Aop))
    ratio = float(np.max(err / (s + 1e-300)))
    assert ratio <= 2.0 ** -14, ratio
    return ratio


PASS_CASES = [
    # m, n, l: ragged tails, tiles split over many CTAs, one-k-block tiles, tall / wide, N = 16 .. 128
    (300, 200, 30),
    (1000, 700, 120),
    (1001, 777, 37),
    (5000, 32, 16),
    (4096, 4096, 128),
    (257, 3000, 8),
    (129, 4100, 80),
]


@pytest.mark.parametrize("m,n,l", PASS_CASES)
@pytest.mark.parametrize("direction", ["ax", "aty"])
def test_pass_parity_tf32x3(m, n, l, direction):
    rng = np.random.default_rng(m + 3 * n)
    # rows of different magnitudes, values with all 24 significant bits in use
    A = (_gauss(71 + m, m, n) * np.exp(rng.uniform(-4, 4, (m, 1)))).astype(np.float32).astype(np.float64)
    Ad = _dev(A)
    K = n if direction == "ax" else m
    olen = m if direction == "ax" else n
    X = _gauss(72 + n, l, K).astype(np.float32).astype(np.float64)
    Ct = corutv.skinny_pass(direction, Ad, _st(X, K), l, mma="tf32x3")
    info = corutv.info_wait()
    assert info.status == 0, corutv.status_string(info.status)
    Aop = A.T if direction == "ax" else A
    ref = O.gemm(X, Aop)
    got = Ct[:, :olen].double().cpu().numpy()
    ratio = _check(got, ref, X, Aop, K)
    print(f"tf32x3 {direction} {m}x{n} l={l}: max err / s = {ratio:.3e} (2^{np.log2(ratio + 1e-300):.1f})")
    # nothing beyond the l x len output was written
    assert torch.count_nonzero(Ct[:, olen:]).item() == 0


@pytest.mark.parametrize("direction", ["ax", "aty"])
def test_tf32x3_far_more_accurate_than_tf32(direction):
    """Relative Frobenius error of the product against FP64: at least 30x below that
    of the TF32 pass on the same inputs (printed beside the FP32 CUDA-core pass's)."""
    m, n, l = 3000, 2500, 96
    A = _gauss(81, m, n).astype(np.float32).astype(np.float64)
    Ad = _dev(A)
    K = n if direction == "ax" else m
    X = _gauss(82, l, K).astype(np.float32).astype(np.float64)
    Xt = _st(X, K)
    ref = O.gemm(X, A.T if direction == "ax" else A)
    olen = ref.shape[1]
    err = {}
    for mma in ("tf32x3", "simt", "tf32"):
        got = corutv.skinny_pass(direction, Ad, Xt, l, mma=mma)[:, :olen].double().cpu().numpy()
        err[mma] = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(err)
    assert err["tf32x3"] < err["tf32"] / 30, err


def test_tf32x3_unbiased_and_deterministic():
    """Positive products (no cancellation): the mean relative error is ~0 (a
    truncating or dropped term would show as a systematic shrink), and two runs
    give identical bits."""
    m, n, l = 2048, 4096, 32
    A = np.abs(_gauss(83, m, n)).astype(np.float32).astype(np.float64)
    Ad = _dev(A)
    X = np.abs(_gauss(84, l, n)).astype(np.float32).astype(np.float64)
    Xt = _st(X, n)
    ref = O.gemm(X, A.T)
    c1 = corutv.skinny_pass("ax", Ad, Xt, l, mma="tf32x3").clone()
    c2 = corutv.skinny_pass("ax", Ad, Xt, l, mma="tf32x3")
    assert torch.equal(c1, c2)
    rel = float(np.mean(c1[:, :m].double().cpu().numpy() / ref - 1.0))
    print(f"tf32x3 mean relative error of positive products (K = {n}): {rel:.3e}")
    assert abs(rel) < 1e-5, rel


def test_tf32x3_fused_fro2():
    """||A||_F^2 fused into the first tf32x3 pass of a solve (FP32 squares per
    stage, FP64 across stages and CTAs)."""
    m, n, l = 3000, 2000, 40
    A = _gauss(85, m, n).astype(np.float32).astype(np.float64)
    Ad = _dev(A)
    phi = torch.tensor(_gauss(86, n, l), dtype=torch.float32, device="cuda")
    r = corutv.solve(Ad, phi, 10, l, 0, mma="tf32x3", want_fro2=True)
    assert r.info.status == 0
    a2 = float(np.sum(A * A))
    assert abs(r.info.fro2_A - a2) <= 1e-6 * a2
