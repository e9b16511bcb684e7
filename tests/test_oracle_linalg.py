"""Pins of the oracle's dense kernels against closed forms, invariants,
brute force and an independent library (numpy/LAPACK SVD)."""
import numpy as np
import pytest

from oracle import corutv_oracle as O
from synth import workloads as W


def test_house_reflects_onto_e1():
    rng = np.random.default_rng(1)
    for x in (rng.standard_normal(7), -np.abs(rng.standard_normal(5)), np.array([0.0, 3.0, 4.0])):
        v, beta, alpha = O.house(x)
        H = np.eye(len(x)) - beta * np.outer(v, v)
        y = H @ x
        assert abs(abs(alpha) - np.linalg.norm(x)) < 1e-14
        assert abs(y[0] - alpha) < 1e-13 and np.abs(y[1:]).max() < 1e-13
        assert np.abs(H @ H.T - np.eye(len(x))).max() < 1e-14
    v, beta, alpha = O.house(np.zeros(4))
    assert beta == 0.0 and alpha == 0.0


@pytest.mark.parametrize("m,l", [(50, 8), (9, 9), (300, 40)])
def test_householder_qr_reconstructs_and_gram_identity(m, l):
    C = np.random.default_rng(m + l).standard_normal((m, l))
    Q, R = O.householder_qr(C)
    assert Q.shape == (m, l) and R.shape == (l, l)
    assert np.abs(Q @ R - C).max() < 1e-13 * np.abs(C).max() * l
    assert O.orthonormality_error(Q) < 1e-14 * l
    assert np.all(np.diag(R) >= 0) and np.abs(np.tril(R, -1)).max() == 0.0
    # R^T R = C^T C (Cholesky factor of the Gram matrix, unique with diag > 0)
    G = C.T @ C
    assert np.abs(R.T @ R - G).max() < 1e-13 * np.abs(G).max()
    L = np.linalg.cholesky(G)            # independent library factorisation
    assert np.abs(L.T - R).max() < 1e-10 * np.abs(R).max()


def test_householder_qr_special_cases():
    rng = np.random.default_rng(3)
    # already orthonormal input -> Q = C, R = I
    Q0, _ = np.linalg.qr(rng.standard_normal((20, 5)))
    Q, R = O.householder_qr(Q0)
    s = np.sign(np.sum(Q * Q0, axis=0))
    assert np.all(s == 1.0)
    assert np.abs(Q - Q0).max() < 1e-14 and np.abs(R - np.eye(5)).max() < 1e-14
    # [R0; 0] with positive diagonal -> Q = [I; 0], R = R0
    R0 = np.triu(rng.standard_normal((4, 4))) + 5 * np.eye(4)
    C = np.vstack([R0, np.zeros((6, 4))])
    Q, R = O.householder_qr(C)
    assert np.abs(R - R0).max() < 1e-14 and np.abs(Q[:4] - np.eye(4)).max() < 1e-15
    # rank-deficient input: Q still orthonormal, QR still C
    C = rng.standard_normal((30, 3)) @ rng.standard_normal((3, 6))
    Q, R = O.householder_qr(C)
    assert O.orthonormality_error(Q) < 1e-14 and np.abs(Q @ R - C).max() < 1e-13


def test_qrcp_worked_2x2():
    # D = [[1, 3], [0, 4]]: column norms 1 and 5 -> column 1 first.
    # (3,4)/5 -> R00 = 5, R01 = 0.6, R11 = 0.8, Q = [[.6, .8], [.8, -.6]]
    D = np.array([[1.0, 3.0], [0.0, 4.0]])
    Q, R, perm = O.qrcp(D)
    assert list(perm) == [1, 0]
    assert np.abs(R - np.array([[5.0, 0.6], [0.0, 0.8]])).max() < 1e-15
    assert np.abs(Q - np.array([[0.6, 0.8], [0.8, -0.6]])).max() < 1e-15


def test_qrcp_invariants():
    rng = np.random.default_rng(5)
    D = rng.standard_normal((12, 12)) * np.logspace(0, -6, 12)[None, :]
    Q, R, perm = O.qrcp(D)
    assert sorted(perm) == list(range(12))
    assert np.abs(D[:, perm] - Q @ R).max() < 1e-14
    assert O.orthonormality_error(Q) < 1e-14
    d = np.diag(R)
    assert np.all(d >= 0) and np.all(np.diff(d) <= 1e-15)
    assert abs(d[0] - np.linalg.norm(D, axis=0).max()) < 1e-14     # first pivot = largest column
    # Businger-Golub: each |R_jj| dominates the trailing column norms of R at step j
    for j in range(12):
        assert d[j] >= np.linalg.norm(R[j:, j:], axis=0).max() - 1e-14


def test_qrcp_diagonal_and_ties():
    D = np.diag([0.5, -3.0, 2.0, 1.0])
    Q, R, perm = O.qrcp(D)
    assert list(perm) == [1, 2, 3, 0]
    assert np.allclose(np.diag(R), [3.0, 2.0, 1.0, 0.5])
    Q, R, perm = O.qrcp(np.eye(5))       # all norms tie -> lowest index each step
    assert list(perm) == [0, 1, 2, 3, 4] and np.allclose(Q, np.eye(5)) and np.allclose(R, np.eye(5))


def test_jacobi_closed_forms():
    s = O.jacobi_svd(np.diag([3.0, -7.0, 0.5, 0.0]))
    assert np.allclose(s, [7.0, 3.0, 0.5, 0.0], atol=1e-15)
    a, b, c, d = 2.0, -1.0, 0.5, 3.0
    s = O.jacobi_svd(np.array([[a, b], [c, d]]))
    assert abs(s[0] * s[1] - abs(a * d - b * c)) < 1e-13
    assert abs(s[0] ** 2 + s[1] ** 2 - (a * a + b * b + c * c + d * d)) < 1e-13
    rng = np.random.default_rng(9)
    U, _ = np.linalg.qr(rng.standard_normal((30, 10)))
    V, _ = np.linalg.qr(rng.standard_normal((10, 10)))
    sig = np.logspace(0, -9, 10)
    s = O.jacobi_svd(U @ np.diag(sig) @ V.T)
    assert np.abs(s - sig).max() < 1e-14


@pytest.mark.parametrize("shape", [(40, 25), (25, 40), (64, 64)])
def test_jacobi_vs_lapack_and_vectors(shape):
    M = np.random.default_rng(sum(shape)).standard_normal(shape)
    s = O.jacobi_svd(M)
    assert np.abs(s - np.linalg.svd(M, compute_uv=False)).max() < 5e-15 * s[0] * max(shape)
    U, s2, V = O.jacobi_svd(M, vectors=True)
    assert np.abs((U * s2) @ V.T - M).max() < 5e-15 * s[0] * max(shape)
    assert O.orthonormality_error(V) < 1e-13


def test_pinv_penrose_conditions():
    rng = np.random.default_rng(11)
    M = rng.standard_normal((9, 3)) @ rng.standard_normal((3, 7))
    P = O.pinv(M)
    assert np.abs(M @ P @ M - M).max() < 1e-12
    assert np.abs(P @ M @ P - P).max() < 1e-12
    assert np.abs((M @ P).T - M @ P).max() < 1e-12
    assert np.abs((P @ M).T - P @ M).max() < 1e-12


# ---------------------------------------------------------------- QLP of the core
def _gapped(c=0, n=60):
    U = W.haar_orthonormal(300 + c, n, n)
    V = W.haar_orthonormal(400 + c, n, n)
    s = np.concatenate([np.linspace(1, 0.5, 20), 1e-3 * np.linspace(1, 0.5, n - 20)])
    return (U * s) @ V.T, s


def test_qlp_structure_and_reconstruction():
    D, s = _gapped()
    Q, L, Wm, perm, Qh = O.qlp(D)
    assert np.linalg.norm(Q @ L @ Wm.T - D) < 1e-13 * np.linalg.norm(D)
    assert np.all(np.triu(L, 1) == 0.0) and np.all(np.diag(L) >= 0.0)
    for M in (Q, Wm, Qh):
        assert np.abs(M.T @ M - np.eye(len(s))).max() < 1e-13
    P = np.eye(len(s))[:, perm]
    assert np.allclose(Wm, P @ Qh, atol=1e-15)


@pytest.mark.parametrize("c", [0, 1, 2])
def test_qlp_tracks_singular_values(c):
    """Stewart's QLP property: the diagonal of L approximates the singular values far
    better than the diagonal of the QRCP's R, and reveals the gap at least as sharply."""
    D, s = _gapped(c)
    _, R, _ = O.qrcp(D)
    _, L, _, _, _ = O.qlp(D)
    dr = np.abs(np.diag(R)) / s
    dl = np.abs(np.diag(L)) / s
    assert np.mean(np.abs(dl - 1)) < 0.5 * np.mean(np.abs(dr - 1))
    assert 0.7 < dl.min() and dl.max() < 1.4
    assert L[19, 19] / L[20, 20] > R[19, 19] / R[20, 20]


def test_qlp_planted_mistake_qr_of_R():
    """Planted mistake: the second QR taken of R instead of R^T does not reproduce D."""
    D, s = _gapped()
    Q, R, perm = O.qrcp(D)
    Qh, Rh = O.householder_qr(R)                 # wrong: should be R^T
    P = np.eye(len(s))[:, perm]
    assert np.linalg.norm(Q @ Rh.T @ (P @ Qh).T - D) > 1e-3 * np.linalg.norm(D)
