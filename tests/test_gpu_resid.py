"""GPU parity of the spectral readout corutv_residual_norm2 (e_k,2 of
Sec. VI-B) with the oracle's power iteration on the same operator: the same
A, U, T, V (the GPU solve's factors, promoted to FP64) and the same start
vector.  FP64: the two iterations differ only in the order of FP64 sums
(bound 1e-10 relative).  FP32: the GPU stores its iterates in FP32 (relative
perturbations ~6e-8 per step, which power iteration does not amplify) and
forms A x with compensated sums before subtracting the low-rank part in FP64,
so the estimates agree to 1e-5 relative.  Converged estimates are also
checked against the largest singular value of the explicit residual."""
import numpy as np
import pytest

from oracle import corutv_oracle as O
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1810_07323_gb300 import corutv


def _factors(r):
    return r.U, r.T, r.V


@pytest.mark.parametrize("k", [20, 30])
def test_fp64_residual_norm2(k):
    d = W.config1()
    A = torch.tensor(d.A, dtype=torch.float64, device="cuda")
    P = torch.tensor(W.phi(1500, 30), dtype=torch.float64, device="cuda")
    r = corutv.solve(A, P, 20, 30, 1)
    x0 = np.random.default_rng(11).standard_normal(1500)
    X0 = torch.tensor(x0, dtype=torch.float64, device="cuda")
    U, T, V = _factors(r)
    for iters in (0, 3, 40):
        g = corutv.residual_norm2(A, U, T, V, X0, k=k, iters=iters)
        o = O.spectral_residual(d.A, U.cpu().numpy(), T.cpu().numpy(), V.cpu().numpy(), k=k, iters=iters, x0=x0)
        assert abs(g - o) < 1e-10 * o, (iters, g, o)
    # converged: the largest singular value of the explicit residual
    R = d.A - O.rank_k(U.cpu().numpy(), T.cpu().numpy(), V.cpu().numpy(), k)
    s = np.linalg.svd(R, compute_uv=False)[0]
    g = corutv.residual_norm2(A, U, T, V, X0, k=k, iters=300)
    assert g <= s * (1 + 1e-12) and g > s * (1 - 1e-3), (g, s)


@pytest.mark.parametrize("k", [100, 120])
def test_fp32_residual_norm2(k):
    g2 = W.config2()
    A64 = g2.block(0, 4000, 0, 3000)
    A = torch.tensor(A64, dtype=torch.float32, device="cuda")
    P = torch.tensor(W.phi(20000, 120)[:3000], dtype=torch.float32, device="cuda")
    r = corutv.solve(A, P, 100, 120, 1)
    x0 = np.random.default_rng(12).standard_normal(3000).astype(np.float32)
    X0 = torch.tensor(x0, device="cuda")
    U, T, V = _factors(r)
    Ah = A.double().cpu().numpy()
    Uh, Th, Vh = U.double().cpu().numpy(), T.cpu().numpy(), V.double().cpu().numpy()
    for iters in (0, 5, 30):
        g = corutv.residual_norm2(A, U, T, V, X0, k=k, iters=iters)
        o = O.spectral_residual(Ah, Uh, Th, Vh, k=k, iters=iters, x0=x0.astype(np.float64))
        print(f"k={k} iters={iters}: gpu {g:.9e} oracle {o:.9e}")
        assert abs(g - o) < 1e-5 * o, (iters, g, o)


def test_residual_norm2_bad_args():
    A = torch.zeros((64, 48), dtype=torch.float32, device="cuda")
    U = torch.zeros((64, 8), dtype=torch.float32, device="cuda")
    V = torch.zeros((48, 8), dtype=torch.float32, device="cuda")
    T = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    x0 = torch.ones(48, dtype=torch.float32, device="cuda")
    assert corutv.residual_norm2(A, U, T, V, x0, iters=4) == 0.0          # R = 0
    with pytest.raises(corutv.CorutvError):
        corutv.residual_norm2(A, U, T, V, x0, k=9)                        # k > l
    with pytest.raises(corutv.CorutvError):
        corutv.residual_norm2(A.bfloat16(), U.bfloat16(), T, V.bfloat16(), x0.bfloat16())   # F32 / F64 only
    with pytest.raises(TypeError):
        corutv.residual_norm2(A, U.double(), T, V, x0)                    # one dtype
