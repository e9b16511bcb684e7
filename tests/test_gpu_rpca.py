"""ALM-CoRUTV robust PCA on the GPU (corutv_rpca, Alg. 5) against the FP64
oracle on the Sec. VI-C synthetic data, through the C ABI.

Both sides take the same M (the FP32 values, promoted to FP64 on the oracle
side), the same Psi and the same schedule parameters (lambda = 1/sqrt(n),
mu_0 = 1.25 / ||M||_2 computed here in FP64, rho = 1.5, mu_bar = 1e7 mu_0).
Tolerances: with FP32 products (mma AUTO, the default for this call) every
iteration's factors agree with the oracle's to ~1e-6 relative, the ranks and
the support of S agree exactly and the recovered L, S to 1e-4 of their norms.
With TF32 passes each CoR-UTV carries ~2^-11 relative product errors; the
stopping rule is still met, the support of S still recovered, and L is checked
to 1e-2 (its rank may exceed the true one by noise directions)."""
import numpy as np
import pytest
import torch

from oracle import rpca_oracle as R
from paper_1810_07323_gb300 import corutv
from synth import counter as C
from synth import workloads as W

pytestmark = pytest.mark.gpu


def _problem(n, sparse, c=6):
    M, L0, S0 = W.rpca_synthetic(n, 0.05, sparse, c=c)
    M = M.astype(np.float32)
    r0 = int(round(0.05 * n))
    l = r0 + 2
    phi = C.normal_block_np(C.stream_seed(2006, 1), l, 0, n, 0, l).astype(np.float32)
    M64 = M.astype(np.float64)
    mu0 = 1.25 / np.linalg.norm(M64, 2)
    return M, M64, L0, S0, r0, l, phi, dict(lam=1.0 / np.sqrt(n), mu0=mu0, rho=1.5, mu_bar=1e7 * mu0)


@pytest.mark.parametrize("mma,ltol", [("auto", 1e-4), ("simt", 1e-4)])
@pytest.mark.parametrize("sparse", [0.05, 0.10])
def test_rpca_parity(mma, ltol, sparse):
    M, M64, L0, S0, r0, l, phi, prm = _problem(500, sparse)
    ref = R.alm_corutv(M64, phi.astype(np.float64), r0, l, 1, prm["lam"], prm["mu0"], prm["rho"], prm["mu_bar"],
                       1e-5, 60)
    Md = torch.tensor(M, device="cuda")
    Pd = torch.tensor(phi, device="cuda")
    out = corutv.rpca(Md, Pd, r0, l, 1, prm["lam"], prm["mu0"], prm["rho"], prm["mu_bar"], 1e-5, 60, mma=mma)
    info = out.info
    assert info.converged == 1 and info.zeta < 1e-5
    assert info.rank == ref["rank"] == r0
    assert abs(info.iters - ref["iters"]) <= 1
    L = out.L.double().cpu().numpy()
    S = out.S.double().cpu().numpy()
    assert np.linalg.norm(L - ref["L"]) < ltol * np.linalg.norm(ref["L"])
    assert np.linalg.norm(S - ref["S"]) < ltol * np.linalg.norm(ref["S"])
    assert np.array_equal(np.abs(S) > 1e-2, np.abs(ref["S"]) > 1e-2)
    # the reconstruction the stopping rule measures, recomputed here
    zeta = np.linalg.norm(M64 - L - S) / np.linalg.norm(M64)
    assert zeta < 2e-5


def test_rpca_tf32_passes():
    M, M64, L0, S0, r0, l, phi, prm = _problem(500, 0.05)
    ref = R.alm_corutv(M64, phi.astype(np.float64), r0, l, 1, prm["lam"], prm["mu0"], prm["rho"], prm["mu_bar"],
                       1e-5, 60)
    out = corutv.rpca(torch.tensor(M, device="cuda"), torch.tensor(phi, device="cuda"), r0, l, 1, prm["lam"],
                      prm["mu0"], prm["rho"], prm["mu_bar"], 1e-5, 60, mma="tf32")
    info = out.info
    L = out.L.double().cpu().numpy()
    S = out.S.double().cpu().numpy()
    errL = np.linalg.norm(L - ref["L"]) / np.linalg.norm(ref["L"])
    print(f"tf32: iters {info.iters} (oracle {ref['iters']}), rank {info.rank}, zeta {info.zeta:.2e}, "
          f"L rel. error vs oracle {errL:.2e}")
    assert info.converged == 1 and info.zeta < 1e-5
    assert r0 <= info.rank <= l
    assert errL < 1e-2
    assert np.array_equal(np.abs(S) > 1.0, np.abs(ref["S"]) > 1.0)


def test_rpca_rejects_bad_arguments():
    M, M64, L0, S0, r0, l, phi, prm = _problem(200, 0.05)
    Md = torch.tensor(M, device="cuda")
    Pd = torch.tensor(phi, device="cuda")
    with pytest.raises(corutv.CorutvError):
        corutv.rpca(Md, Pd, r0, l, 1, prm["lam"], -1.0, prm["rho"], prm["mu_bar"])        # mu_0 > 0
    with pytest.raises(corutv.CorutvError):
        corutv.rpca(Md, Pd, r0, l, 1, prm["lam"], prm["mu0"], 0.5, prm["mu_bar"])         # rho >= 1
    with pytest.raises(corutv.CorutvError):
        corutv.rpca(Md, Pd, r0, 200, 1, prm["lam"], prm["mu0"], prm["rho"], prm["mu_bar"])  # l < min(m, n)
