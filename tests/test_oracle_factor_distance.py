"""Pins of the factor-space parity measure rho = ||U1 T1 V1^T - U2 T2 V2^T||_F /
||U2 T2 V2^T||_F (`factor_distance`), the number every GPU parity test asserts on.

It is pinned to things outside itself: the explicitly formed difference of the two
products (brute force), closed forms for planted perturbations of known size, the
invariances the measure exists for (column signs of a UTV factorisation and the
pivot permutation), agreement of its two branches, and planted mistakes that these
pins catch."""
import numpy as np
import pytest

from oracle import corutv_oracle as O


def _orth(rng, rows, cols):
    Q, R = np.linalg.qr(rng.standard_normal((rows, cols)))
    return Q * np.sign(np.diag(R))


def _utv(seed, m, n, l, triangular=True):
    """A random UTV factorisation: orthonormal U (m x l), V (n x l), T (l x l)."""
    rng = np.random.default_rng(seed)
    U = _orth(rng, m, l)
    V = _orth(rng, n, l)
    T = rng.standard_normal((l, l))
    if triangular:
        T = np.triu(T)
    return U, T, V


def _explicit(U1, T1, V1, U2, T2, V2):
    X1 = U1 @ T1 @ V1.T
    X2 = U2 @ T2 @ V2.T
    return np.linalg.norm(X1 - X2) / np.linalg.norm(X2)


def _perpendicular(rng, Q):
    """A unit vector orthogonal to range(Q)."""
    w = rng.standard_normal(Q.shape[0])
    w -= Q @ (Q.T @ w)
    w -= Q @ (Q.T @ w)
    return w / np.linalg.norm(w)


# ------------------------------------------------------------------ brute force, both branches
@pytest.mark.parametrize("m,n,l", [(40, 30, 8), (300, 200, 20), (600, 520, 60)])
def test_matches_explicit_difference(m, n, l):
    """Against the explicitly formed ||X1 - X2||_F / ||X2||_F for two unrelated
    factorisations and for two that differ by a small random perturbation
    (joint-basis branch: m, n >= 2 l)."""
    U1, T1, V1 = _utv(1, m, n, l)
    U2, T2, V2 = _utv(2, m, n, l)
    assert O.factor_distance(U1, T1, V1, U2, T2, V2) == pytest.approx(_explicit(U1, T1, V1, U2, T2, V2), rel=1e-12)
    rng = np.random.default_rng(3)
    U3 = U1 + 1e-6 * rng.standard_normal(U1.shape)
    V3 = V1 + 1e-6 * rng.standard_normal(V1.shape)
    T3 = T1 + 1e-6 * np.triu(rng.standard_normal(T1.shape))
    ref = _explicit(U3, T3, V3, U1, T1, V1)
    got = O.factor_distance(U3, T3, V3, U1, T1, V1)
    assert 1e-7 < ref < 1e-4
    assert got == pytest.approx(ref, rel=1e-8)


@pytest.mark.parametrize("m,n,l", [(50, 30, 20), (35, 60, 20)])
def test_explicit_branch_matches_explicit_difference(m, n, l):
    """When 2 l exceeds a dimension the function forms the products itself: the
    same value as brute force."""
    U1, T1, V1 = _utv(4, m, n, l)
    rng = np.random.default_rng(5)
    T2 = T1 + 1e-3 * np.triu(rng.standard_normal(T1.shape))
    assert O.factor_distance(U1, T2, V1, U1, T1, V1) == pytest.approx(_explicit(U1, T2, V1, U1, T1, V1), rel=1e-10)


def test_branches_agree():
    """The two branches on the same products: a factorisation whose U has fewer
    than 2 l rows (explicit branch) against the same factorisation with U padded by
    zero rows to more than 2 l rows (joint-basis branch).  Zero rows leave U
    orthonormal and the products unchanged up to those rows, so rho must agree."""
    l = 30
    U1, T1, V1 = _utv(6, 120, 100, l)
    rng = np.random.default_rng(7)
    T2 = T1 + 0.1 * np.triu(rng.standard_normal(T1.shape))
    small_m = 2 * l - 1
    Us1 = _orth(rng, small_m, l)
    Us2 = _orth(rng, small_m, l)
    expl = O.factor_distance(Us1, T1, V1, Us2, T2, V1)
    assert expl == pytest.approx(_explicit(Us1, T1, V1, Us2, T2, V1), rel=1e-12)
    pad = np.zeros((2 * l + 7 - small_m, l))
    joint = O.factor_distance(np.vstack([Us1, pad]), T1, V1, np.vstack([Us2, pad]), T2, V1)
    assert expl == pytest.approx(joint, rel=1e-11)


# ------------------------------------------------------------------ closed forms
@pytest.mark.parametrize("eps", [1e-12, 1e-7, 1e-3, 0.5])
def test_planted_core_perturbation(eps):
    """T2 = T1 + eps E with the same orthonormal U, V: U (T1 - T2) V^T has norm
    eps ||E||_F, so rho = eps ||E||_F / ||T2||_F exactly."""
    U, T1, V = _utv(8, 400, 300, 25)
    E = np.triu(np.random.default_rng(9).standard_normal(T1.shape))
    T2 = T1 + eps * E
    want = eps * np.linalg.norm(E) / np.linalg.norm(T2)
    got = O.factor_distance(U, T1, V, U, T2, V)
    assert abs(got - want) <= 1e-12 * want + 1e-15


@pytest.mark.parametrize("theta", [1e-9, 1e-5, 1e-2, 0.7])
@pytest.mark.parametrize("side", ["U", "V"])
def test_planted_rotation(theta, side):
    """Column j of U (or V) rotated by theta towards a unit vector w outside the
    basis: the columns stay orthonormal, the changed column moves by
    2 sin(theta/2), so rho = 2 sin(theta/2) ||T(j,:)|| / ||T||_F (U) or
    2 sin(theta/2) ||T(:,j)|| / ||T||_F (V)."""
    U, T, V = _utv(10, 500, 350, 20)
    rng = np.random.default_rng(11)
    j = 3
    if side == "U":
        w = _perpendicular(rng, U)
        U2 = U.copy()
        U2[:, j] = np.cos(theta) * U[:, j] + np.sin(theta) * w
        got = O.factor_distance(U2, T, V, U, T, V)
        want = 2 * np.sin(theta / 2) * np.linalg.norm(T[j, :]) / np.linalg.norm(T)
    else:
        w = _perpendicular(rng, V)
        V2 = V.copy()
        V2[:, j] = np.cos(theta) * V[:, j] + np.sin(theta) * w
        got = O.factor_distance(U, T, V2, U, T, V)
        want = 2 * np.sin(theta / 2) * np.linalg.norm(T[:, j]) / np.linalg.norm(T)
    assert abs(got - want) <= 1e-12 * want + 1e-15


# ------------------------------------------------------------------ invariances
def test_invariant_to_signs_and_pivots():
    """rho = 0 (to rounding) between a factorisation and its re-signed and
    re-pivoted forms: U S with S T (S = diag(+-1)), T S' with V S', and T P
    with V P for a permutation P all leave U T V^T unchanged."""
    m, n, l = 300, 260, 24
    U, T, V = _utv(12, m, n, l)
    rng = np.random.default_rng(13)
    s1 = np.where(rng.random(l) < 0.5, -1.0, 1.0)
    s2 = np.where(rng.random(l) < 0.5, -1.0, 1.0)
    P = rng.permutation(l)
    U2 = U * s1
    T2 = (s1[:, None] * T) * s2[None, :]
    V2 = V * s2
    T2, V2 = T2[:, P], V2[:, P]
    assert O.factor_distance(U2, T2, V2, U, T, V) < 1e-14
    assert O.factor_distance(U, T, V, U2, T2, V2) < 1e-14
    # on an oracle solve: its perm applied to the unpermuted basis reproduces V
    A = U @ np.diag(np.linspace(1, 0.01, l)) @ V.T
    r = O.corutv(A, np.random.default_rng(14).standard_normal((n, l)), 10, l, 0)
    Q2, perm = r["Q2"], r["perm"]
    Tunperm = np.empty_like(r["T"])
    Tunperm[:, perm] = r["T"]
    assert O.factor_distance(r["U"], Tunperm, Q2, r["U"], r["T"], r["V"]) < 1e-13


def test_symmetric_scale_and_zero_distance():
    """rho(X, X) = 0; rho scales as the definition says when the reference is scaled."""
    U, T, V = _utv(15, 200, 150, 10)
    assert O.factor_distance(U, T, V, U, T, V) == 0.0
    # X1 = 2 X2: ||X1 - X2|| / ||X2|| = 1; X1 = X2 / 2: 1/2
    assert O.factor_distance(U, 2 * T, V, U, T, V) == pytest.approx(1.0, rel=1e-13)
    assert O.factor_distance(U, 0.5 * T, V, U, T, V) == pytest.approx(0.5, rel=1e-13)


# ------------------------------------------------------------------ planted mistakes
def _joint_basis_distance(U1, T1, V1, U2, T2, V2, qu_from, qv_from, drop_term=False):
    """The joint-basis computation with its bases taken from the given blocks
    (a faithful copy of the measure when qu_from = [U1 U2], qv_from = [V1 V2])."""
    Qu, _ = O.householder_qr(qu_from)
    Qv, _ = O.householder_qr(qv_from)
    X1 = O.gemm(O.gemm(O.gemm(Qu.T, U1), T1), O.gemm(V1.T, Qv))
    X2 = O.gemm(O.gemm(O.gemm(Qu.T, U2), T2), O.gemm(V2.T, Qv))
    if drop_term:
        return float(np.linalg.norm(X1) / np.linalg.norm(X2) - 1.0)
    return float(np.linalg.norm(X1 - X2) / np.linalg.norm(X2))


def test_planted_mistakes_are_caught(monkeypatch):
    """Mistakes that would make every parity test pass vacuously: a joint basis
    built from one factorisation only (a rotation out of its span is projected
    away), and the norm of the wrong term (|‖X1‖ - ‖X2‖| instead of ‖X1 - X2‖,
    blind to rotations).  Each fails the rotation closed form; the faithful copy
    passes it."""
    U, T, V = _utv(16, 500, 350, 20)
    rng = np.random.default_rng(17)
    theta, j = 1e-3, 2
    w = _perpendicular(rng, U)
    U2 = U.copy()
    U2[:, j] = np.cos(theta) * U[:, j] + np.sin(theta) * w
    want = 2 * np.sin(theta / 2) * np.linalg.norm(T[j, :]) / np.linalg.norm(T)
    ok = _joint_basis_distance(U2, T, V, U, T, V, np.hstack([U2, U]), np.hstack([V, V]))
    assert abs(ok - want) <= 1e-12 * want
    one_sided = _joint_basis_distance(U2, T, V, U, T, V, U, np.hstack([V, V]))
    assert abs(one_sided - want) > 0.1 * want
    wrong_term = _joint_basis_distance(U2, T, V, U, T, V, np.hstack([U2, U]), np.hstack([V, V]), drop_term=True)
    assert abs(wrong_term - want) > 0.1 * want
    # and the oracle function itself, with its QR made to return only the first block's basis
    orig = O.householder_qr

    def first_block_only(C):
        Q, R = orig(C)
        half = C.shape[1] // 2
        Q = Q.copy()
        Q[:, half:] = 0.0
        return Q, R

    monkeypatch.setattr(O, "householder_qr", first_block_only)
    broken = O.factor_distance(U, T, V, U2, T, V)
    monkeypatch.undo()
    fixed = O.factor_distance(U, T, V, U2, T, V)
    assert abs(fixed - want) <= 1e-12 * want
    assert abs(broken - want) > 0.1 * want
