"""QLP of the core on the GPU (factor = QLP: the QRCP of D, then an unpivoted
QR of R~^T) against the FP64 oracle's QLP, through the C ABI.

Tolerances as for the QRCP form (the second factorisation adds one more
FP32 Householder pass of an l x l block): FP32 products rho <= 1e-4, TF32
rho <= 1e-3; T is lower triangular (RIGHT) or upper (LEFT) exactly, with a
non-negative diagonal; diag(T) matches the oracle's L to 1e-4 relative (FP32
products) where the pivots agree.
"""
import numpy as np
import pytest

from oracle import corutv_oracle as O
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1810_07323_gb300 import corutv


def _decay(m, n, c, rank=60):
    U = W.haar_orthonormal(500 + c, m, rank)
    V = W.haar_orthonormal(600 + c, n, rank)
    s = np.exp(-np.arange(rank) / 8.0)
    return (U * s) @ V.T


def _solve(A, phi, k, l, q, mma, side="right", factor="qlp"):
    m, n = A.shape
    lda = -(-n // 8) * 8
    Ad = torch.zeros((m, lda), dtype=torch.float32, device="cuda")[:, :n]
    Ad.copy_(torch.tensor(A, device="cuda").float())
    Pd = torch.tensor(phi, device="cuda").float()
    r = corutv.solve(Ad, Pd, k, l, q, side=side, mma=mma, factor=factor, want_fro2=True)
    assert r.info.status == 0
    return r, Ad.double().cpu().numpy(), Pd.double().cpu().numpy()


@pytest.mark.parametrize("mma,tol", [("simt", 1e-4), ("auto", 1e-3)])
@pytest.mark.parametrize("m,n,k,l,q,side", [(1200, 800, 20, 40, 1, "right"), (3000, 2000, 60, 120, 0, "right"),
                                            (500, 900, 10, 24, 1, "left")])
def test_qlp_parity(mma, tol, m, n, k, l, q, side):
    A = _decay(m, n, 1)
    phi = W.phi(m if side == "left" else n, l, c=11)
    r, A64, P64 = _solve(A, phi, k, l, q, mma, side)
    ref = O.corutv(A64, P64, k, l, q, side=side, factor="qlp")
    U, T, V = r.U.double().cpu().numpy(), r.T.cpu().numpy(), r.V.double().cpu().numpy()
    rho = O.factor_distance(U, T, V, ref["U"], ref["T"], ref["V"])
    assert rho < tol, rho
    off = np.triu(T, 1) if side == "right" else np.tril(T, -1)
    assert np.abs(off).max() == 0.0 and np.all(np.diag(T) >= 0.0)
    assert O.orthonormality_error(U) < 5e-5 and O.orthonormality_error(V) < 5e-5
    if mma == "simt":
        d, dref = np.diag(T), np.diag(ref["T"])
        assert np.abs(d[:k] - dref[:k]).max() < 1e-4 * dref[0]
    # readouts: ||T||_F^2 of the returned T and the rank-k part T(1:k, :) (RIGHT: L(1:k, 1:k))
    assert abs(r.info.fro2_T - float(np.sum(T ** 2))) < 1e-5 * r.info.fro2_T
    if side == "right":
        assert abs(r.info.fro2_Tk - float(np.sum(T[:k, :k] ** 2))) < 1e-5 * r.info.fro2_T


def test_qlp_same_product_as_qrcp():
    """The QLP and QRCP forms factor the same core: their U T V^T agree to FP32 rounding."""
    A = _decay(1500, 1000, 2)
    phi = W.phi(1000, 48, c=12)
    r1, _, _ = _solve(A, phi, 30, 48, 1, "simt", factor="qrcp")
    r2, _, _ = _solve(A, phi, 30, 48, 1, "simt", factor="qlp")
    f = lambda r: (r.U.double().cpu().numpy(), r.T.cpu().numpy(), r.V.double().cpu().numpy())
    assert O.factor_distance(*f(r2), *f(r1)) < 1e-5


def test_qlp_f64_unsupported():
    A = torch.zeros((300, 200), dtype=torch.float64, device="cuda")
    P = torch.zeros((200, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(corutv.CorutvError):
        corutv.solve(A, P, 5, 10, 0, factor="qlp")
