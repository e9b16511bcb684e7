"""Pins of the CoR-UTV oracle against what the paper and the mathematics fix:
exact recovery, singular values when rank(A) <= l, structure of U, T, V, the
Pythagorean identity of the exact core, the core identity, Eckart-Young
floors, interlacing, the valid rank-revealing inequalities, the Fig. 1
statistics, and planted mistakes that these pins must catch."""
import os

import numpy as np
import pytest

from oracle import corutv_oracle as O
from synth import workloads as W


@pytest.fixture(scope="module")
def cfg1():
    return W.config1()


@pytest.fixture(scope="module")
def cfg1_exact():
    return W.config1(exact_rank=True)


def _small_decay(m=160, n=120, c=3):
    """Small matrix with a known, decaying spectrum."""
    U = W.haar_orthonormal(101 + c, m, n)
    V = W.haar_orthonormal(202 + c, n, n)
    s = np.exp(-np.arange(n) / 6.0)
    return (U * s) @ V.T, s


@pytest.mark.parametrize("q", [0, 1])
@pytest.mark.parametrize("l", [20, 30])
def test_exact_recovery_rank_k(cfg1_exact, q, l):
    """Thm. 4 with A_0 = 0 and range inclusion: a rank-k A is recovered exactly for l >= k."""
    A = cfg1_exact.A
    r = O.corutv(A, W.phi(A.shape[1], l), 20, l, q)
    rel = O.fro_residual(A, r["U"], r["T"], r["V"]) / np.linalg.norm(A)
    assert rel < 1e-13
    # sigma_j(T) = sigma_j(A) when rank(A) <= l (T is a unitary compression of A)
    sT = O.jacobi_svd(r["T"])
    assert np.abs(sT[:20] - cfg1_exact.sigma[:20]).max() < 1e-13
    if l > 20:
        assert sT[20:].max() < 1e-13


def test_structure(cfg1):
    A = cfg1.A
    r = O.corutv(A, W.phi(1500, 30), 20, 30, 0)
    U, T, V, perm = r["U"], r["T"], r["V"], r["perm"]
    assert O.orthonormality_error(U) < 1e-14 * 30
    assert O.orthonormality_error(V) < 1e-14 * 30
    assert np.abs(np.tril(T, -1)).max() == 0.0
    d = np.diag(T)
    assert np.all(d >= 0) and np.all(np.diff(d) <= 0)
    assert sorted(perm) == list(range(30))
    assert np.array_equal(V, r["Q2"][:, perm])          # V = Q2 P~
    assert abs(d[0] - np.linalg.norm(r["D"], axis=0).max()) < 1e-14


@pytest.mark.parametrize("q", [0, 2])
def test_pythagorean_identity(cfg1, q):
    """Exact core: U^T A V = Q~^T D P~ = T, hence ||A - U T V^T||_F^2 = ||A||_F^2 - ||T||_F^2,
    and the same for the rank-k view with T(1:k, :)."""
    A = cfg1.A
    r = O.corutv(A, W.phi(1500, 30), 20, 30, q)
    a2 = np.linalg.norm(A) ** 2
    e2 = O.fro_residual(A, r["U"], r["T"], r["V"]) ** 2
    assert abs(e2 - (a2 - np.linalg.norm(r["T"]) ** 2)) < 1e-12 * a2
    ek2 = O.fro_residual(A, r["U"], r["T"], r["V"], k=20) ** 2
    assert abs(ek2 - (a2 - np.linalg.norm(r["T"][:20]) ** 2)) < 1e-12 * a2
    assert np.abs(r["U"].T @ A @ r["V"] - r["T"]).max() < 1e-13


def test_core_identity_literal(cfg1):
    """Literal Alg. 2 (q = 0): C2 = A^T C1 = A^T Q1 R1 = Q2 R2, so
    D = Q1^T A Q2 = (Q2 R2 R1^-1)^T Q2 = R1^-T R2^T."""
    A = cfg1.A
    r = O.corutv(A, W.phi(1500, 30), 20, 30, 0, orth="literal")
    Dref = np.linalg.solve(r["R1"].T, r["R2"].T)
    assert np.abs(r["D"] - Dref).max() < 1e-9 * np.abs(r["D"]).max()


def test_approx_core_equals_exact_core(cfg1):
    """Q1^T A lies in range(Q2)^T (C2 is A^T times the last C1), so
    D_approx = Q1^T C1 (Q2^T C2_prev)^+ reproduces D exactly (Eq. (D_approx))."""
    A = cfg1.A
    for q in (0, 1):
        re = O.corutv(A, W.phi(1500, 30), 20, 30, q)
        ra = O.corutv(A, W.phi(1500, 30), 20, 30, q, core="approx")
        assert np.abs(re["D"] - ra["D"]).max() < 1e-9


def test_stabilised_equals_literal():
    """Intermediate orthonormalisation multiplies the literal iterate by an
    invertible triangular factor: same Q1, Q2 (hence same factors) when the
    literal iterate is still well conditioned."""
    A, s = _small_decay()
    phi = W.phi(120, 12)
    rs = O.corutv(A, phi, 8, 12, 1)
    rl = O.corutv(A, phi, 8, 12, 1, orth="literal")
    assert np.abs(rs["Q1"] - rl["Q1"]).max() < 1e-8
    assert np.abs(rs["Q2"] - rl["Q2"]).max() < 1e-8
    assert O.factor_distance(rs["U"], rs["T"], rs["V"], rl["U"], rl["T"], rl["V"]) < 1e-8


@pytest.mark.parametrize("q", [0, 1, 2])
def test_eckart_young_floors_interlacing_and_rank_revealing(q):
    A, s = _small_decay()
    k, l = 10, 16
    r = O.corutv(A, W.phi(120, l, c=7), k, l, q)
    sA = O.jacobi_svd(A)
    assert np.abs(sA - s).max() < 1e-13                   # brute-force SVD of the constructed A
    eF = O.fro_residual(A, r["U"], r["T"], r["V"], k=k)
    e2 = O.spectral_residual(A, r["U"], r["T"], r["V"], k=k)
    assert eF >= np.sqrt(np.sum(sA[k:] ** 2)) * (1 - 1e-12)
    assert e2 >= sA[k] * (1 - 1e-6)
    sD = O.jacobi_svd(r["D"])
    assert np.all(sD <= sA[:l] * (1 + 1e-12))              # sigma_j(D) <= sigma_j(A)
    T = r["T"]
    assert O.jacobi_svd(T[:k, :k])[-1] <= sD[k - 1] * (1 + 1e-12)   # sigma_min(T11) <= sigma_k(D)
    assert O.jacobi_svd(T[k:, k:])[0] >= sD[k] * (1 - 1e-12)        # ||T22||_2 >= sigma_{k+1}(D)
    # power iterations only improve the rank-k error here
    if q:
        r0 = O.corutv(A, W.phi(120, l, c=7), k, l, 0)
        assert eF <= O.fro_residual(A, r0["U"], r0["T"], r0["V"], k=k) * (1 + 1e-9)


def test_theorem2_style_bound_on_exact_low_rank_plus_tail():
    """Thm. 2/Thm. 4 structure: for A = A_k + A_0 the CoR-UTV error is at most
    ||A_0|| plus terms that vanish as the tail shrinks; with q = 1 the rank-l
    error must approach the optimum sigma_{l+1} (Sec. VI-B1)."""
    A, s = _small_decay()
    l = 16
    r = O.corutv(A, W.phi(120, l, c=9), 10, l, 1)
    e2 = O.spectral_residual(A, r["U"], r["T"], r["V"])
    assert e2 <= 3.0 * s[l]


def test_fig1_statistics(golden_dir):
    """Fig. 1 (Sec. VI-A): mean |T_jj| over 20 trials on NoisyLowRank-I
    (order 1000, k = 20, l = 40, q = 0) against the printed CoR-UTV curve, and
    the generator's SVD against the printed SVD curve.  Only statistics are
    pinned: the paper's random draws are not reproducible."""
    tab = np.loadtxt(os.path.join(golden_dir, "fig1_noisylowrank1.txt"))
    sig_paper, cor_paper = tab[:, 1], tab[:, 2]
    d = W.noisy_lowrank(1000, 20, 0.01)
    sv = np.linalg.svd(d.A, compute_uv=False)[:40]        # library SVD: checks the generator only
    assert np.abs(sv[:20] / sig_paper[:20] - 1).max() < 0.01
    assert np.abs(sv[20:] / sig_paper[20:] - 1).max() < 0.05
    T = [np.diag(O.corutv(d.A, W.phi(1000, 40, trial=t), 20, 40, 0)["T"]) for t in range(20)]
    mean = np.mean(np.abs(T), axis=0)
    assert np.abs(mean[:20] / cor_paper[:20] - 1).max() < 0.01
    assert np.abs(mean[20:] / cor_paper[20:] - 1).max() < 0.05
    # the gap at k = 20 is revealed
    assert mean[19] / mean[20] > 100


def test_side_left_is_ulv(cfg1):
    """Sec. III m < n modification: run on A^T; T lower triangular."""
    A = cfg1.A
    rl = O.corutv(A, W.phi(2000, 30), 20, 30, 0, side="left")
    assert np.abs(np.triu(rl["T"], 1)).max() == 0.0
    rt = O.corutv(A.T, W.phi(2000, 30), 20, 30, 0)
    assert np.array_equal(rl["U"], rt["V"]) and np.array_equal(rl["T"], rt["T"].T)
    a2 = np.linalg.norm(A) ** 2
    assert abs(O.fro_residual(A, rl["U"], rl["T"], rl["V"]) ** 2 - (a2 - np.linalg.norm(rl["T"]) ** 2)) < 1e-12 * a2


def test_argument_checks():
    A = np.zeros((10, 8))
    with pytest.raises(ValueError):
        O.corutv(A, np.zeros((8, 8)), 2, 8, 0)          # l < min(m, n)
    with pytest.raises(ValueError):
        O.corutv(A, np.zeros((8, 4)), 5, 4, 0)          # k <= l
    with pytest.raises(ValueError):
        O.corutv(A, np.zeros((8, 4)), 2, 4, -1)         # q >= 0


# ------------------------------------------------------------------ planted mistakes
def test_planted_transposed_permutation_is_caught(cfg1):
    """Reading Alg. 2's printed V = Q2 P~^T instead of V = Q2 P~ breaks the
    reconstruction pin (this is why V = Q2 P~ is the reading)."""
    A = cfg1.A
    r = O.corutv(A, W.phi(1500, 30), 20, 30, 0)
    inv = np.argsort(r["perm"])
    assert not np.array_equal(inv, r["perm"])
    Vbad = r["Q2"][:, inv]
    a2 = np.linalg.norm(A) ** 2
    good = O.fro_residual(A, r["U"], r["T"], r["V"]) ** 2
    bad = O.fro_residual(A, r["U"], r["T"], Vbad) ** 2
    assert abs(good - (a2 - np.linalg.norm(r["T"]) ** 2)) < 1e-12 * a2
    assert abs(bad - (a2 - np.linalg.norm(r["T"]) ** 2)) > 1e-3 * a2


def test_planted_wrong_sign_householder_is_caught(monkeypatch):
    """A Householder vector with the wrong sign (v0 = x0 + alpha reflects x
    onto -alpha e1 while alpha is recorded as R_jj) fails the QR pins."""
    orig = O.house

    def bad_house(x):
        v, beta, alpha = orig(x)
        v = x.copy()
        v[0] = x[0] + alpha
        nv = np.dot(v, v)
        return v, (2.0 / nv if nv > 0 else 0.0), alpha

    monkeypatch.setattr(O, "house", bad_house)
    C = np.random.default_rng(2).standard_normal((20, 5))
    Q, R = O.householder_qr(C)
    assert np.abs(Q @ R - C).max() > 1e-3


def test_correction_core_is_projection_of_reference(cfg1):
    """Correction pass (core from A_core): with A_core = A it is the plain exact core;
    otherwise T is the compression U^T A_core V, the Pythagorean identity holds for
    A_core, and for the fixed bases no other core (in particular the one from the
    perturbed A) leaves a smaller residual of A_core (D = Q1^T A_core Q2 minimises
    ||A_core - Q1 D Q2^T||_F)."""
    from oracle import precision as P
    A = cfg1.A
    Phi = W.phi(1500, 30)
    r0 = O.corutv(A, Phi, 20, 30, 1)
    r1 = O.corutv(A, Phi, 20, 30, 1, A_core=A)
    assert np.array_equal(r0["T"], r1["T"]) and np.array_equal(r0["U"], r1["U"])
    vals, sc = P.quantize_fp8(A.astype(np.float32))
    Aq = P.dequantize_fp8(vals, sc)
    assert np.linalg.norm(Aq - A) > 1e-3 * np.linalg.norm(A)        # a real perturbation
    rc = O.corutv(Aq, Phi, 20, 30, 1, A_core=A)
    ru = O.corutv(Aq, Phi, 20, 30, 1)
    assert np.abs(rc["U"].T @ A @ rc["V"] - rc["T"]).max() < 1e-13
    a2 = np.linalg.norm(A) ** 2
    e2 = O.fro_residual(A, rc["U"], rc["T"], rc["V"]) ** 2
    assert abs(e2 - (a2 - np.linalg.norm(rc["T"]) ** 2)) < 1e-12 * a2
    assert np.allclose(rc["Q1"], ru["Q1"]) and np.allclose(rc["Q2"], ru["Q2"])   # same range finding
    e_u = np.linalg.norm(A - ru["Q1"] @ ru["D"] @ ru["Q2"].T)
    e_c = np.linalg.norm(A - rc["Q1"] @ rc["D"] @ rc["Q2"].T)
    assert e_c <= e_u
    with pytest.raises(ValueError):
        O.corutv(Aq, Phi, 20, 30, 1, core="approx", A_core=A)


@pytest.mark.parametrize("q", [0, 1])
def test_qlp_core_same_product(cfg1, q):
    """factor="qlp" factors the same core: U T V^T is the QRCP form's product (to rounding),
    T is lower triangular with a non-negative diagonal and U, V stay orthonormal."""
    A = cfg1.A
    phi = W.phi(A.shape[1], 30)
    r1 = O.corutv(A, phi, 20, 30, q)
    r2 = O.corutv(A, phi, 20, 30, q, factor="qlp")
    assert O.factor_distance(r2["U"], r2["T"], r2["V"], r1["U"], r1["T"], r1["V"]) < 1e-13
    assert np.all(np.triu(r2["T"], 1) == 0.0) and np.all(np.diag(r2["T"]) >= 0.0)
    assert O.orthonormality_error(r2["U"]) < 1e-13 and O.orthonormality_error(r2["V"]) < 1e-13


def test_qlp_exact_recovery(cfg1_exact):
    A = cfg1_exact.A
    r = O.corutv(A, W.phi(A.shape[1], 25), 20, 25, 0, factor="qlp")
    assert O.fro_residual(A, r["U"], r["T"], r["V"]) / np.linalg.norm(A) < 1e-13


def _gapped(m=90, n=60, c=11):
    """A with sigma = 10, 9, ..., 6 (five), then 1, 0.5, 0.25, ...: a rank-5 view leaves
    a residual whose top two singular values are about 1 and 0.5 (power iteration converges
    like 0.25^iters)."""
    U = W.haar_orthonormal(301 + c, m, n)
    V = W.haar_orthonormal(302 + c, n, n)
    s = np.concatenate([np.arange(10.0, 5.0, -1.0), 0.5 ** np.arange(n - 5)])
    return (U * s) @ V.T


@pytest.mark.parametrize("k", [5, 8])
def test_spectral_residual_power_iteration(k):
    """The spectral readout against the largest singular value of the explicitly formed
    residual R = A - U(:,1:k) T(1:k,:) V^T (Jacobi SVD and LAPACK): converged after enough
    steps, a lower bound after any number of steps, and the start vector only sets the
    path.  A residual formed with all l rows of T (a dropped truncation) gives another value."""
    A = _gapped()
    l = 8
    r = O.corutv(A, W.phi(60, l, c=5), 5, l, 1)
    R = A - O.rank_k(r["U"], r["T"], r["V"], k)
    s_exact = O.jacobi_svd(R)[0]
    assert abs(s_exact - np.linalg.svd(R, compute_uv=False)[0]) < 1e-12 * s_exact
    x0 = np.random.default_rng(3).standard_normal(60)
    est = O.spectral_residual(A, r["U"], r["T"], r["V"], k=k, iters=200, x0=x0)
    assert abs(est - s_exact) < 1e-10 * s_exact
    for it in (0, 1, 3):
        e = O.spectral_residual(A, r["U"], r["T"], r["V"], k=k, iters=it, x0=x0)
        assert e <= s_exact * (1 + 1e-12)
    # y = R x0 / ||x0|| after zero steps
    assert abs(O.spectral_residual(A, r["U"], r["T"], r["V"], k=k, iters=0, x0=x0)
               - np.linalg.norm(R @ x0) / np.linalg.norm(x0)) < 1e-12 * s_exact
    est_seed = O.spectral_residual(A, r["U"], r["T"], r["V"], k=k, iters=200, seed=9)
    assert abs(est_seed - s_exact) < 1e-10 * s_exact
    if k < l:
        full = O.spectral_residual(A, r["U"], r["T"], r["V"], k=None, iters=200, x0=x0)
        assert abs(full - s_exact) > 1e-3 * s_exact
