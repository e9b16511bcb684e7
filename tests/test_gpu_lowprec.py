"""GPU parity of the low-precision storage modes of A (BF16, FP8 e4m3 with
128 x 128 tile scales) through the C ABI: the quantiser bit for bit against
oracle/precision.py, the kind::f16 tensor-core passes against the FP64 product
of the dequantised A, the fused ||A||_F^2, and whole solves (with and without
the FP32 correction pass) against the FP64 oracle run on the same stored
values.

Pass bounds.  A in BF16 (or FP8 dequantised with a power-of-two scale) is
exact in BF16; the FP32 sketch operand x is split x = x_hi + x_lo + d with
x_hi = bf16(x), x_lo = bf16(x - x_hi), |d| <= 2^-18 |x|; BF16 x BF16 products
are exact in FP32 and 2K of them are accumulated in FP32.  Hence
  |C - C_ref| <= (2^-18 + (2K + 8) 2^-23) (|X| |A|)        (deterministic)
with a factor 2 of slack on the accumulation.  The rounding errors are
independent and zero-mean, so against the natural scale
s = sqrt((X o X)(A o A)) they stay near 2^-18 + 2^-24 sqrt(K); the test asks
max |C - C_ref| / s <= 2^-13, which a pass that dropped x_lo (errors ~2^-10 s)
fails.  A non-power-of-two FP8 scale adds one BF16 rounding of the dequantised
value: 2^-9 |X| |A| more in the deterministic bound.
"""
import numpy as np
import pytest

from oracle import corutv_oracle as O
from oracle import precision as P
from synth import counter as C
from synth import workloads as W

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


def _dev(vals, dtype):
    """Device copy of host values already representable in `dtype`, rows padded
    to a 16-byte-multiple pitch with lda > n."""
    m, n = vals.shape
    lda = -(-n // 16) * 16 + 16
    buf = torch.zeros((m, lda), dtype=dtype, device="cuda")[:, :n]
    buf.copy_(torch.tensor(np.asarray(vals, dtype=np.float32)).to(dtype).cuda())
    return buf


def _stored(A32, kind):
    """(device A, device scales or None, FP64 dequantised A) from the oracle's conversion."""
    if kind == "bf16":
        v = P.bf16_round(A32)
        return _dev(v, torch.bfloat16), None, v.astype(np.float64)
    vals, sc = P.quantize_fp8(A32)
    return _dev(vals, torch.float8_e4m3fn), torch.tensor(sc, dtype=torch.float32, device="cuda"), \
        P.dequantize_fp8(vals, sc)


PASS_CASES = [
    (300, 200, 30),
    (1000, 700, 120),
    (1001, 777, 37),
    (5000, 48, 16),
    (4096, 4096, 128),
    (257, 3000, 8),
]


def _check_pass(got, ref, X, Aop, K, extra_rel=0.0):
    err = np.abs(got - ref)
    det = (2.0 ** -18 + (2 * K + 8) * 2.0 ** -23 + extra_rel) * (np.abs(X) @ np.abs(Aop))
    assert np.all(err <= det + 1e-30), float(np.max(err / (det + 1e-300)))
    if extra_rel == 0.0:
        s = np.sqrt((X * X) @ (Aop * Aop))
        ratio = float(np.max(err / (s + 1e-300)))
        assert ratio <= 2.0 ** -13, ratio


@pytest.mark.parametrize("m,n,l", PASS_CASES)
@pytest.mark.parametrize("direction", ["ax", "aty"])
@pytest.mark.parametrize("kind", ["bf16", "fp8"])
def test_pass_parity_lowprec(m, n, l, direction, kind):
    rng = np.random.default_rng(m * 7 + n)
    # rows of very different magnitudes: exercises the per-tile FP8 scales
    A32 = (_gauss(31 + m, m, n) * np.exp(rng.uniform(-3, 3, (m, 1)))).astype(np.float32)
    Ad, S, Adq = _stored(A32, kind)
    K = n if direction == "ax" else m
    olen = m if direction == "ax" else n
    X = _gauss(32 + n, l, K).astype(np.float32).astype(np.float64)
    Ct = corutv.skinny_pass(direction, Ad, _st(X, K), l, mma="bf16x2", a_tile_scales=S)
    info = corutv.info_wait()
    assert info.status == 0, corutv.status_string(info.status)
    Aop = Adq.T if direction == "ax" else Adq
    ref = O.gemm(X, Aop)
    got = Ct[:, :olen].double().cpu().numpy()
    _check_pass(got, ref, X, Aop, K)
    assert torch.count_nonzero(Ct[:, olen:]).item() == 0


@pytest.mark.parametrize("direction", ["ax", "aty"])
def test_pass_fp8_arbitrary_scales(direction):
    """Scales that are not powers of two: the dequantised value is rounded once to BF16."""
    m, n, l = 700, 520, 24
    vals, _ = P.quantize_fp8(_gauss(41, m, n).astype(np.float32))
    sc = np.exp(np.random.default_rng(5).uniform(-2, 2, (-(-m // 128), -(-n // 128)))).astype(np.float32)
    Ad = _dev(vals, torch.float8_e4m3fn)
    Adq = P.dequantize_fp8(vals, sc.astype(np.float64))
    K = n if direction == "ax" else m
    X = _gauss(42, l, K).astype(np.float32).astype(np.float64)
    Ct = corutv.skinny_pass(direction, Ad, _st(X, K), l, mma="bf16x2",
                            a_tile_scales=torch.tensor(sc, device="cuda"))
    Aop = Adq.T if direction == "ax" else Adq
    got = Ct[:, :(m if direction == "ax" else n)].double().cpu().numpy()
    _check_pass(got, O.gemm(X, Aop), X, Aop, K, extra_rel=2.0 ** -9 * (1 + 2.0 ** -7))


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
def test_pass_lowprec_deterministic(kind):
    m, n, l = 3000, 2000, 64
    Ad, S, _ = _stored(_gauss(1, m, n).astype(np.float32), kind)
    for direction in ("ax", "aty"):
        K = n if direction == "ax" else m
        Xt = _st(_gauss(2, l, K), K)
        c1 = corutv.skinny_pass(direction, Ad, Xt, l, mma="bf16x2", a_tile_scales=S).clone()
        c2 = corutv.skinny_pass(direction, Ad, Xt, l, mma="bf16x2", a_tile_scales=S)
        assert torch.equal(c1, c2)


def test_pass_lowprec_alignment():
    """FP8 rows need a 16-byte pitch for TMA: an explicit bf16x2 pass refuses
    lda = n + 1 (ERR_ALIGN); AUTO falls back to the SIMT pass."""
    m, n, l = 256, 300, 16
    vals, sc = P.quantize_fp8(_gauss(3, m, n).astype(np.float32))
    buf = torch.zeros((m, n + 1), dtype=torch.float8_e4m3fn, device="cuda")[:, :n]
    buf.copy_(torch.tensor(vals.astype(np.float32)).to(torch.float8_e4m3fn).cuda())
    S = torch.tensor(sc, dtype=torch.float32, device="cuda")
    Xt = _st(_gauss(4, l, n), n)
    with pytest.raises(corutv.CorutvError) as e:
        corutv.skinny_pass("ax", buf, Xt, l, mma="bf16x2", a_tile_scales=S)
    assert e.value.status == corutv.ERR_ALIGN
    Ct = corutv.skinny_pass("ax", buf, Xt, l, mma="auto", a_tile_scales=S)
    ref = O.gemm(_gauss(4, l, n).astype(np.float32).astype(np.float64), P.dequantize_fp8(vals, sc).T)
    got = Ct[:, :m].double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-6


# ---------------------------------------------------------------------------- quantiser
@pytest.mark.parametrize("m,n", [(300, 260), (1000, 1000), (129, 4097), (5, 7)])
def test_quantize_matches_oracle(m, n):
    rng = np.random.default_rng(m + n)
    A32 = (_gauss(50 + m, m, n) * np.exp(rng.uniform(-8, 8, (m, 1)))).astype(np.float32)
    if m >= 256 and n >= 256:
        A32[128:256, 128:256] = 0.0            # an all-zero tile: scale 1
    Ad = torch.tensor(A32, device="cuda")
    qb, _ = corutv.quantize(Ad, "bf16")
    assert np.array_equal(qb.float().cpu().numpy(), P.bf16_round(A32))
    q8, S = corutv.quantize(Ad, "fp8")
    vals, sc = P.quantize_fp8(A32)
    assert np.array_equal(S.double().cpu().numpy(), sc)
    assert np.array_equal(q8.double().cpu().numpy(), vals)


# ---------------------------------------------------------------------------- solves
TOL_LP = 1e-4     # same arithmetic after the passes as the FP32 SIMT path; pass errors ~2^-18


@pytest.fixture(scope="module")
def cfg1():
    return W.config1()


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
@pytest.mark.parametrize("q", [0, 2])
@pytest.mark.parametrize("small_f64", [False, True])
def test_solve_lowprec_parity(cfg1, kind, q, small_f64):
    """small_f64: the Gram reductions, Cholesky factors, core and QRCP in FP64."""
    A32 = cfg1.A.astype(np.float32)
    Ad, S, Adq = _stored(A32, kind)
    phi = W.phi(A32.shape[1], 30).astype(np.float32)
    r = corutv.solve(Ad, torch.tensor(phi, device="cuda"), 20, 30, q, a_tile_scales=S, want_fro2=True,
                     small_f64=small_f64)
    assert r.info.status == 0
    U, T, V = r.U.double().cpu().numpy(), r.T.cpu().numpy(), r.V.double().cpu().numpy()
    ref = O.corutv(Adq, phi.astype(np.float64), 20, 30, q)
    rho = O.factor_distance(U, T, V, ref["U"], ref["T"], ref["V"])
    print(f"config1 {kind} q={q} small_f64={small_f64}: rho={rho:.3e}")
    assert rho < TOL_LP, rho
    a2 = float(np.sum(Adq ** 2))
    assert abs(r.info.fro2_A - a2) < 1e-6 * a2
    assert r.info.passes_over_A == 2 * q + 3


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
@pytest.mark.parametrize("side", ["right", "left"])
@pytest.mark.parametrize("small_f64", [False, True])
def test_solve_corrected_parity(kind, side, small_f64):
    """FP32 correction pass: range finding on the stored A, core from the FP32 A
    (small_f64: Gram reductions, Cholesky, core and QRCP in FP64)."""
    g = W.config3(m=2048, n=1536)
    A32 = g.block(0, g.m, 0, g.n).astype(np.float32)
    if side == "left":
        A32 = np.ascontiguousarray(A32.T)
    m, n = A32.shape
    Ad, S, Adq = _stored(A32, kind)
    phi = W.phi(m if side == "left" else n, 80).astype(np.float32)
    Aref = torch.tensor(A32, device="cuda")
    r = corutv.solve(Ad, torch.tensor(phi, device="cuda"), 64, 80, 2, side=side, a_tile_scales=S, A_ref=Aref,
                     want_fro2=True, small_f64=small_f64)
    assert r.info.status == 0
    U, T, V = r.U.double().cpu().numpy(), r.T.cpu().numpy(), r.V.double().cpu().numpy()
    ref = O.corutv(Adq, phi.astype(np.float64), 64, 80, 2, side=side, A_core=A32.astype(np.float64))
    rho = O.factor_distance(U, T, V, ref["U"], ref["T"], ref["V"])
    print(f"config3-like {kind} {side} corrected small_f64={small_f64}: rho={rho:.3e}")
    # the correction pass runs on the FP32-class split-operand tensor-core engine (TF32X3)
    assert rho < 1e-4, rho
    A64 = A32.astype(np.float64)
    a2 = float(np.sum(A64 ** 2))
    assert abs(r.info.fro2_A - a2) < 1e-6 * a2
    assert r.info.passes_over_A == 2 * 2 + 3
    # T is the compression of the FP32 matrix: Pythagorean identity on A_ref
    e2 = O.fro_residual(A64, U, T, V) ** 2
    assert abs(e2 - (a2 - np.sum(T ** 2))) < 6e-4 * a2
