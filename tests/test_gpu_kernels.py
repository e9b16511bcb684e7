"""GPU parity of each step of the hot path, called through the C ABI, against
the FP64 oracle on the same seeded inputs: the streaming passes (Sec. III
products, both directions, every engine), Gram reductions, shifted
CholeskyQR orthonormalisation, the QRCP of the core, and ||A||_F^2."""
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


def _st(host, ld_len, dtype):
    """Skinny-transposed device copy (l rows, leading dimension ld_for(len))."""
    l, n = host.shape
    buf = torch.zeros((l, corutv.ld_for(ld_len)), dtype=dtype, device="cuda")
    buf[:, :n] = torch.tensor(host, dtype=dtype, device="cuda")
    return buf


# ---------------------------------------------------------------------------- passes
PASS_CASES = [
    # m, n, l : ragged tails, tiles split across many CTAs, single-k-block tiles, tall/wide
    (300, 200, 30),
    (1000, 700, 120),
    (1001, 777, 37),
    (5000, 32, 16),
    (4096, 4096, 128),
    (257, 3000, 8),
]


def _tf32_bound(A, X, mode):
    # TF32 operands keep 10 explicit mantissa bits.  Truncated by the tensor core
    # ("tf32t"): |a b - t(a) t(b)| <= (2^-10 + 2^-10 + 2^-20) |a b|.  Rounded to nearest
    # first ("tf32"): <= (2^-11 + 2^-11 + 2^-22) |a b|.  FP32 accumulation adds at most
    # K u32 |a| |b|, well inside the 0.25-0.5 x 2^-10 slack left here.
    c = 2.5 if mode == "tf32t" else 1.25
    return c * 2.0 ** -10 * (np.abs(A) @ np.abs(X))


@pytest.mark.parametrize("m,n,l", PASS_CASES)
@pytest.mark.parametrize("direction", ["ax", "aty"])
@pytest.mark.parametrize("eng", ["f64-simt", "f32-simt", "f32-tf32", "f32-tf32t", "bf16-simt"])
def test_pass_parity(m, n, l, direction, eng):
    dt_name, mma = eng.split("-")
    dt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dt_name]
    cdt = torch.float64 if dt_name == "f64" else torch.float32
    # rows padded to a 16-byte pitch (lda > n) so every engine can read them
    lda = -(-n // 8) * 8 + 8
    A_dev = torch.zeros((m, lda), dtype=dt, device="cuda")[:, :n]
    A_dev.copy_(torch.tensor(_gauss(11 + m, m, n), dtype=torch.float64, device="cuda").to(dt))
    K = n if direction == "ax" else m
    olen = m if direction == "ax" else n
    X = _gauss(22 + n, l, K)
    Xt = _st(X, K, cdt)
    Ct = corutv.skinny_pass(direction, A_dev, Xt, l, mma=mma)
    info = corutv.info_wait()
    assert info.status == 0, corutv.status_string(info.status)
    A64 = A_dev.double().cpu().numpy()
    X64 = Xt[:, :K].double().cpu().numpy()
    ref = O.gemm(X64, A64.T) if direction == "ax" else O.gemm(X64, A64)     # (l x olen)
    got = Ct[:, :olen].double().cpu().numpy()
    if mma in ("tf32", "tf32t"):
        bound = _tf32_bound(X64, A64.T if direction == "ax" else A64, mma)
        assert np.all(np.abs(got - ref) <= bound + 1e-30)
    else:
        tol = 1e-13 if dt_name == "f64" else 2e-6
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < tol, err
    # nothing beyond the l x len output was written
    assert torch.count_nonzero(Ct[:, olen:]).item() == 0


def test_pass_fp8_tile_scales():
    m, n, l = 300, 260, 20
    A = _gauss(5, m, n)
    sc = np.abs(A).reshape(1, -1).max() / 448.0
    ntr, ntc = -(-m // 128), -(-n // 128)
    scales = np.full((ntr, ntc), sc, dtype=np.float32)
    scales[1, 1] = sc * 2
    q = A.copy()
    for i in range(ntr):
        for j in range(ntc):
            q[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128] /= scales[i, j]
    A8 = torch.tensor(q, dtype=torch.float32, device="cuda").to(torch.float8_e4m3fn)
    S = torch.tensor(scales, device="cuda")
    X = _gauss(6, l, n)
    Ct = corutv.skinny_pass("ax", A8, _st(X, n, torch.float32), l, mma="simt", a_tile_scales=S)
    deq = A8.float().cpu().numpy().astype(np.float64)
    for i in range(ntr):
        for j in range(ntc):
            deq[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128] *= scales[i, j]
    ref = O.gemm(X, deq.T)
    got = Ct[:, :m].double().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-6


@pytest.mark.parametrize("direction", ["ax", "aty"])
def test_pass_deterministic(direction):
    m, n, l = 3000, 2000, 64
    A = torch.tensor(_gauss(1, m, n), dtype=torch.float32, device="cuda")
    K = n if direction == "ax" else m
    Xt = _st(_gauss(2, l, K), K, torch.float32)
    c1 = corutv.skinny_pass(direction, A, Xt, l, mma="tf32").clone()
    c2 = corutv.skinny_pass(direction, A, Xt, l, mma="tf32")
    assert torch.equal(c1, c2)


def test_rounded_tf32_is_unbiased():
    """Rounding operands to nearest removes the systematic shrink of the
    truncating tensor core: the mean relative error of sum_k x_k a_k over many
    positive products is ~0 with "tf32" and ~ -7e-4 with "tf32t" (each of the
    two truncated operands loses ~3.5e-4 on average)."""
    m, n, l = 2048, 4096, 32
    A = torch.tensor(np.abs(_gauss(3, m, n)), dtype=torch.float32, device="cuda")
    X = np.abs(_gauss(4, l, n))
    Xt = _st(X, n, torch.float32)
    ref = O.gemm(X, A.double().cpu().numpy().T)
    rel = {}
    for mode in ("tf32", "tf32t"):
        got = corutv.skinny_pass("ax", A, Xt, l, mma=mode)[:, :m].double().cpu().numpy()
        rel[mode] = float(np.mean(got / ref - 1.0))
    assert abs(rel["tf32"]) < 2e-5, rel
    assert -1e-3 < rel["tf32t"] < -4e-4, rel


def test_pass_rejects_misaligned_rows():
    A = torch.zeros((64, 66), dtype=torch.float32, device="cuda")[:, :63]   # lda 66 * 4 bytes: not 16-aligned
    Xt = _st(np.zeros((4, 63)), 63, torch.float32)
    with pytest.raises(corutv.CorutvError) as e:
        corutv.skinny_pass("ax", A, Xt, 4, mma="tf32")
    assert e.value.status == corutv.ERR_ALIGN
    # AUTO falls back to the SIMT engine for rows TMA cannot address
    corutv.skinny_pass("ax", A, Xt, 4, mma="auto")


# ---------------------------------------------------------------------------- Gram / orth
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("length,l", [(5000, 120), (333, 17), (40, 40)])
def test_gram_parity(dt, length, l):
    X, Y = _gauss(3, l, length), _gauss(4, l, length)
    G = corutv.gram(_st(X, length, dt), _st(Y, length, dt), length, l).cpu().numpy()
    Xd = torch.tensor(X, dtype=dt).double().numpy()
    Yd = torch.tensor(Y, dtype=dt).double().numpy()
    ref = O.gemm(Xd, Yd.T)
    tol = 1e-14 if dt == torch.float64 else 1e-6
    assert np.abs(G - ref).max() <= tol * np.abs(Xd).sum(1)[:, None].max() * np.abs(Yd).max() * 4 + 1e-300


def _ill_conditioned(length, l, cond, seed):
    Q, _ = np.linalg.qr(_gauss(seed, length, l))
    W, _ = np.linalg.qr(_gauss(seed + 1, l, l))
    s = np.logspace(0, -np.log10(cond), l)
    return ((Q * s) @ W.T).T.copy()          # ST layout (l x length)


@pytest.mark.parametrize("dt,cond,orth_tol", [(torch.float32, 1e4, 5e-6), (torch.float32, 1e6, 5e-6),
                                             (torch.float64, 1e12, 1e-13)])
def test_orthonormalize_ill_conditioned(dt, cond, orth_tol):
    length, l = 20000, 96
    Ct = _ill_conditioned(length, l, cond, 9)
    buf = _st(Ct, length, dt)
    corutv.orthonormalize(buf, length, l)
    Q = buf[:, :length].double().cpu().numpy().T
    assert O.orthonormality_error(Q) < orth_tol
    # same range: the input lies in span(Q).  The residual C - Q Q^T C is the backward
    # error of CholeskyQR, ~ c l u ||C||_F with u the unit roundoff of the arithmetic: at
    # l = 96 and u32 = 6e-8 that is ~6e-6 c, so 2e-5 allows c ~ 3 (FP64: 1e-13, c ~ 5)
    C0 = torch.tensor(Ct, dtype=dt).double().numpy().T
    res = C0 - Q @ (Q.T @ C0)
    assert np.linalg.norm(res) / np.linalg.norm(C0) < (2e-5 if dt == torch.float32 else 1e-13)


@pytest.mark.parametrize("dt,cond", [(torch.float64, 1e8), (torch.float32, 1e3), (torch.float32, 1.0)])
def test_orthonormalize_returns_R(dt, cond):
    """R_out is the product of the three CholeskyQR factors: C = Q R, R upper
    triangular with a positive diagonal (cond 1: the FP32 third pass is skipped)."""
    length, l = 5000, 40
    Ct = _ill_conditioned(length, l, cond, 21)
    buf = _st(Ct, length, dt)
    R = corutv.orthonormalize(buf, length, l, want_R=True).cpu().numpy()
    Q = buf[:, :length].double().cpu().numpy().T
    C0 = torch.tensor(Ct, dtype=dt).double().numpy().T
    assert np.abs(np.tril(R, -1)).max() == 0.0 and np.all(np.diag(R) > 0)
    tol = 1e-13 if dt == torch.float64 else 2e-5
    assert np.linalg.norm(C0 - Q @ R) / np.linalg.norm(C0) < tol
    assert O.orthonormality_error(Q) < (1e-13 if dt == torch.float64 else 5e-6)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_orthonormalize_rank_deficient(dt):
    """A numerically rank-deficient block (rank 20 of 30) still yields an
    orthonormal basis containing its range (any orthonormal completion is
    valid: U T V^T does not depend on it)."""
    length, l = 3000, 30
    B = _gauss(12, length, 20) @ _gauss(13, 20, l)
    buf = _st(B.T.copy(), length, dt)
    corutv.orthonormalize(buf, length, l)
    Q = buf[:, :length].double().cpu().numpy().T
    # CholeskyQR backward error ~ c l u ||C|| (l = 30): 1e-13 in FP64, 2e-5 in FP32
    tol = 1e-13 if dt == torch.float64 else 2e-5
    assert O.orthonormality_error(Q) < tol
    B0 = torch.tensor(B, dtype=dt).double().numpy()
    assert np.linalg.norm(B0 - Q @ (Q.T @ B0)) / np.linalg.norm(B0) < tol


def test_orthonormalize_replaces_zero_columns():
    """Exactly dependent (zero) columns break the unshifted Cholesky: they are
    detected, replaced by pseudo-random columns and orthonormalised (any orthonormal
    completion of the range is correct: U T V^T does not change)."""
    length, l = 2000, 24
    B = _gauss(14, length, l)
    B[:, [3, 11, 20]] = 0.0
    buf = _st(B.T.copy(), length, torch.float64)
    corutv.orthonormalize(buf, length, l)
    info = corutv.info_wait()
    Q = buf[:, :length].cpu().numpy().T
    assert info.chol_fallbacks == 3
    assert O.orthonormality_error(Q) < 1e-13
    assert np.linalg.norm(B - Q @ (Q.T @ B)) / np.linalg.norm(B) < 1e-13


# ---------------------------------------------------------------------------- QRCP
def _qrcp_gpu(D, dtype):
    Q, R, perm, fro2 = corutv.qrcp(torch.tensor(D, dtype=torch.float64, device="cuda"), dtype=dtype)
    return Q.cpu().numpy(), R.cpu().numpy(), perm.cpu().numpy(), fro2.cpu().numpy()


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-5)])
@pytest.mark.parametrize("l", [2, 30, 77, 128])
def test_qrcp_parity(dtype, tol, l):
    rng_D = _gauss(40 + l, l, l) * np.logspace(0, -3, l)[None, :]
    Q, R, perm, fro2 = _qrcp_gpu(rng_D, dtype)
    Qo, Ro, po = O.qrcp(rng_D)
    assert np.array_equal(perm, po)                     # well separated norms: same pivots
    scale = np.abs(Ro).max()
    assert np.abs(R - Ro).max() <= tol * scale * 10
    assert np.abs(Q - Qo).max() <= tol * 10 * l
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.all(np.diag(R) >= 0)
    assert abs(fro2[0] - np.sum(Ro ** 2)) <= tol * np.sum(Ro ** 2) * 10


def test_qrcp_worked_example_and_ties():
    Q, R, perm, _ = _qrcp_gpu(np.array([[1.0, 3.0], [0.0, 4.0]]), "f64")
    assert list(perm) == [1, 0]
    assert np.abs(R - np.array([[5.0, 0.6], [0.0, 0.8]])).max() < 1e-15
    assert np.abs(Q - np.array([[0.6, 0.8], [0.8, -0.6]])).max() < 1e-15
    Q, R, perm, _ = _qrcp_gpu(np.eye(7), "f32")
    assert list(perm) == list(range(7))
    Q, R, perm, _ = _qrcp_gpu(np.diag([0.5, -3.0, 2.0, 1.0]), "f64")
    assert list(perm) == [1, 2, 3, 0]
    assert np.allclose(np.diag(R), [3.0, 2.0, 1.0, 0.5])


def test_qrcp_zero_matrix():
    Q, R, perm, _ = _qrcp_gpu(np.zeros((9, 9)), "f32")
    assert np.all(R == 0) and sorted(perm) == list(range(9))
    assert O.orthonormality_error(Q) < 1e-6


# ---------------------------------------------------------------------------- ||A||_F^2
@pytest.mark.parametrize("dt", [torch.float64, torch.float32, torch.bfloat16])
def test_fro2(dt):
    A = torch.tensor(_gauss(77, 1234, 567), dtype=torch.float64, device="cuda").to(dt)
    got = corutv.fro2(A).item()
    ref = float(np.sum(A.double().cpu().numpy() ** 2))
    assert abs(got - ref) <= (1e-13 if dt == torch.float64 else 1e-6) * ref
