"""Pins of the ALM-CoRUTV oracle (Sec. V, Alg. 5; Sec. VI-C, Tables I and II):
closed forms of the shrinkage and CoR-UTV thresholding operators, exact
recovery by C_delta of a matrix of rank <= l, recovery of the Sec. VI-C
synthetic data with the printed rank, support size and iteration count, and
a planted mistake (the mu update as printed, with max) that the recovery pin
must catch."""
import os

import numpy as np
import pytest

from oracle import corutv_oracle as O
from oracle import rpca_oracle as R
from synth import counter as C
from synth import workloads as W


def _golden(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "tables_I_II_rpca.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t, n, r, s, it, z = line.split()
            rows.append(dict(table=t, n=int(n), rank=int(r), nnz=int(s), iters=int(it), zeta=float(z)))
    return rows


def _params(M, n):
    # lambda = 1/sqrt(max(m, n)), mu_0 = 1.25 / ||M||_2, rho = 1.5, mu_bar = 1e7 mu_0: inputs
    # of Alg. 5 that the paper takes from its reference [LLS2011] without printing them
    mu0 = 1.25 / np.linalg.norm(M, 2)
    return 1.0 / np.sqrt(n), mu0, 1.5, 1e7 * mu0


def _run(n, sparse, mu_update="min", max_iter=60):
    M, L0, S0 = W.rpca_synthetic(n, 0.05, sparse)
    r0 = int(round(0.05 * n))
    l = r0 + 2
    phi = C.normal_block_np(C.stream_seed(2006, 1), l, 0, n, 0, l)
    lam, mu0, rho, mu_bar = _params(M, n)
    out = R.alm_corutv(M, phi, r0, l, 1, lam, mu0, rho, mu_bar, 1e-5, max_iter, mu_update=mu_update)
    return out, M, L0, S0, r0


def test_shrink_closed_form():
    x = np.array([-3.0, -1.0, -0.5, 0.0, 0.5, 1.0, 3.0])
    np.testing.assert_array_equal(R.shrink(x, 1.0), [-2.0, 0.0, 0.0, 0.0, 0.0, 0.0, 2.0])
    np.testing.assert_array_equal(R.shrink(x, 0.0), x)
    assert np.all(R.shrink(x, 10.0) == 0.0)


def test_threshold_exact_for_rank_le_l():
    """rank(B) <= l: CoR-UTV reproduces B exactly, so C_delta(B) = B once delta is below
    every non-zero diagonal of T, and C_delta(B) = 0 once delta is above T_11."""
    rng = np.random.default_rng(5)
    U = np.linalg.qr(rng.standard_normal((300, 6)))[0]
    V = np.linalg.qr(rng.standard_normal((200, 6)))[0]
    B = (U * np.array([9.0, 7.0, 5.0, 3.0, 2.0, 1.0])) @ V.T
    phi = rng.standard_normal((200, 10))
    L, r, f = R.corutv_threshold(B, phi, 6, 10, 0, 1e-6)
    assert r == 6 and np.linalg.norm(L - B) < 1e-12 * np.linalg.norm(B)
    L, r, f = R.corutv_threshold(B, phi, 6, 10, 0, 1.01 * f["T"][0, 0])
    assert r == 0 and not np.any(L)
    # r counts the diagonals above delta (the diagonal is non-increasing)
    d = np.diag(f["T"])
    for delta in (0.5, 1.5, 2.5, 4.0):
        assert R.corutv_threshold(B, phi, 6, 10, 0, delta)[1] == int(np.sum(d > delta))


@pytest.mark.parametrize("sparse,iters_lo,iters_hi", [(0.05, 12, 14), (0.10, 14, 16)])
def test_recovery_sec6c(sparse, iters_lo, iters_hi):
    """Sec. VI-C data at n = 500: L and S recovered (rank r, exact support of S), zeta < 1e-5,
    in about the iteration count of Tables I / II (12 and 14 at n = 1000)."""
    out, M, L0, S0, r0 = _run(500, sparse)
    assert out["zeta"] < 1e-5
    assert out["rank"] == r0
    assert np.linalg.norm(out["L"] - L0) < 1e-4 * np.linalg.norm(L0)
    assert np.array_equal(np.abs(out["S"]) > 1e-3, S0 != 0)
    assert iters_lo <= out["iters"] <= iters_hi


def test_tables_I_II_n1000(golden_dir):
    """The n = 1000 rows of Tables I and II: rank(L*) = 50, ||S*||_0 = s, zeta < 1e-5 and the
    iteration count within one of the printed value."""
    for row in _golden(golden_dir):
        if row["n"] != 1000:
            continue
        out, M, L0, S0, r0 = _run(1000, 0.05 if row["table"] == "I" else 0.10)
        assert out["rank"] == row["rank"]
        nnz = int(np.sum(np.abs(out["S"]) > 1e-3))
        assert abs(nnz - row["nnz"]) <= 0.01 * row["nnz"]
        assert out["zeta"] < 1e-5
        assert abs(out["iters"] - row["iters"]) <= 1


def test_planted_mistake_mu_update_as_printed():
    """The update printed in Alg. 5, mu_{j+1} = max(rho mu_j, mu_bar), jumps to mu_bar after the
    first iteration: the thresholds collapse and S absorbs everything, so the recovery pin fails."""
    out, M, L0, S0, r0 = _run(500, 0.05, mu_update="max")
    assert not (out["rank"] == r0 and np.linalg.norm(out["L"] - L0) < 1e-4 * np.linalg.norm(L0))
