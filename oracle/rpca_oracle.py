"""Plain FP64 CPU oracle for ALM-CoRUTV robust PCA (test infrastructure only).

Imported only by the tests, by `__graft_entry__.smoke()` and by the CPU
baseline leg of `bench.py`; the library never calls it and shares no code
with it.  Everything is float64 numpy on top of the CoR-UTV oracle.

Paper: M. F. Kaloorazi and R. C. de Lamare, "Compressed Randomized UTV
Decompositions for Low-Rank Approximations and Big Data Applications"
(arXiv 1810.07323), Sec. V (robust PCA by ALM, Alg. 4 and the proposed
ALM-CoRUTV, Alg. 5) and Sec. VI-C (synthetic recovery, Tables I and II).

Functions
  shrink            the shrinkage operator S_delta(x) = sgn(x) max(|x| - delta, 0)  (Sec. V)
  corutv_threshold  the CoR-UTV thresholding operator C_delta(B) = U(:,1:r) T(1:r,:) V^T,
                    r = number of diagonals of T greater than delta               (Sec. V, Eq. (C_delta))
  alm_corutv        Alg. 5 (ALM-CoRUTV) with the stopping rule of Sec. VI-C

Readings (where Alg. 5 is garbled or silent; the same readings drive the GPU path):
  - the multiplier update is mu_{j+1} = min(rho mu_j, mu_bar): continuation grows mu
    and mu_bar caps it (the printed max would jump to mu_bar at once);
  - the S step uses Y_j (the printed Y without index);
  - r counts diagonals of T above delta (T's diagonal is non-negative here);
  - one Gaussian test matrix Psi (passed in) serves every iteration's CoR-UTV;
  - lambda, mu_0, mu_bar and rho are inputs (the paper takes them from its
    reference [LLS2011] without printing them).
Pins: tests/test_oracle_rpca.py (closed forms of both operators, exact recovery
by C_delta of a matrix of rank <= l, recovery of the Sec. VI-C synthetic data,
and a planted mistake: the printed max in the mu update fails to recover it).
"""
from __future__ import annotations

import numpy as np

from . import corutv_oracle as O


def shrink(X: np.ndarray, delta: float) -> np.ndarray:
    """S_delta(x) = sgn(x) max(|x| - delta, 0), elementwise (Sec. V)."""
    X = np.asarray(X, dtype=np.float64)
    return np.sign(X) * np.maximum(np.abs(X) - delta, 0.0)


def corutv_threshold(B: np.ndarray, Phi: np.ndarray, k: int, l: int, q: int, delta: float):
    """C_delta(B) = U(:,1:r) T(1:r,:) V^T with r = #{j : T_jj > delta} (Sec. V).

    Returns (L, r, factorisation dict)."""
    f = O.corutv(B, Phi, k, l, q)
    d = np.diag(f["T"])
    r = int(np.sum(d > delta))
    L = O.gemm(O.gemm(f["U"][:, :r], f["T"][:r, :]), f["V"].T) if r > 0 else np.zeros_like(B, dtype=np.float64)
    return L, r, f


def alm_corutv(M: np.ndarray, Phi: np.ndarray, k: int, l: int, q: int, lam: float, mu0: float, rho: float,
               mu_bar: float, tol: float = 1e-5, max_iter: int = 100, mu_update: str = "min") -> dict:
    """Alg. 5 (ALM-CoRUTV), Y_0 = S_0 = 0, stopped when
    ||M - L - S||_F / ||M||_F < tol (Sec. VI-C).  mu_update="max" is the
    update exactly as printed (kept for the planted-mistake pin)."""
    M = np.asarray(M, dtype=np.float64)
    Y = np.zeros_like(M)
    S = np.zeros_like(M)
    mu = float(mu0)
    nM = float(np.linalg.norm(M))
    L = np.zeros_like(M)
    r = 0
    zeta = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        L, r, _ = corutv_threshold(M - S + Y / mu, Phi, k, l, q, 1.0 / mu)   # Alg. 5 step 2
        S = shrink(M - L + Y / mu, lam / mu)                                  # step 3
        R = M - L - S
        Y = Y + mu * R                                                        # step 4
        mu = min(rho * mu, mu_bar) if mu_update == "min" else max(rho * mu, mu_bar)   # step 5
        zeta = float(np.linalg.norm(R)) / nM
        if zeta < tol:
            break
    return dict(L=L, S=S, Y=Y, iters=it, rank=r, zeta=zeta, mu=mu)
