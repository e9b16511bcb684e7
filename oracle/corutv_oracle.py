"""Plain FP64 CPU oracle for CoR-UTV (test infrastructure only).

This module is the yardstick the GPU library is checked against.  It is
imported only by the tests, by `__graft_entry__.smoke()` and by the CPU
baseline leg of `bench.py`; the library itself never calls it, and it shares
no code with the CUDA path.  Everything is float64 numpy; a numpy matrix
product serves as the GEMM primitive, every factorisation is written out.

Paper: M. F. Kaloorazi and R. C. de Lamare, "Compressed Randomized UTV
Decompositions for Low-Rank Approximations and Big Data Applications"
(arXiv 1810.07323).  Citations name its sections, equations and algorithms.

Functions
  householder_qr   thin QR of a tall block, diag(R) >= 0       (Sec. III, QR of C1, C2)
  qrcp             Householder QR with column pivoting           (Sec. III, Eq. (D = Q~ R~ P~^T))
  qlp              QRCP followed by an unpivoted QR of R^T (Stewart's QLP), the core variant
  jacobi_svd       one-sided cyclic Jacobi SVD (quality tool)    (Sec. II, Eq. (SVD))
  corutv           Alg. 2 / Alg. 3, stabilised or literal, exact or approximate core
  rank_k           Sec. VI-B2 rank-k view U(:,1:k) T(1:k,:) V^T
  quality helpers  Frobenius / spectral residuals, factor-space distance

Pins: every function is checked in tests/test_oracle_*.py against closed
forms, invariants, brute force and the paper's Fig. 1 statistics.
Parity unpinned: the paper's own per-trial random draws (only statistics
of its Fig. 1 are pinned).
"""
from __future__ import annotations

import numpy as np

EPS64 = np.finfo(np.float64).eps


# ============================================================================ GEMM
def gemm(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Plain float64 matrix product (library primitive)."""
    return np.asarray(A, dtype=np.float64) @ np.asarray(B, dtype=np.float64)


# ============================================================================ Householder
def house(x: np.ndarray):
    """Householder reflector H = I - beta v v^T with H x = alpha e_1.

    alpha = -sign(x_0) ||x|| (sign(0) taken as +1), v_0 = x_0 - alpha.
    A zero x gives beta = 0 (H = I) and alpha = 0.
    """
    x = np.asarray(x, dtype=np.float64)
    nrm = np.sqrt(np.dot(x, x))
    v = x.copy()
    if nrm == 0.0:
        v[:] = 0.0
        v[0] = 1.0
        return v, 0.0, 0.0
    s = 1.0 if x[0] >= 0.0 else -1.0
    alpha = -s * nrm
    v[0] = x[0] - alpha
    beta = 2.0 / np.dot(v, v)
    return v, beta, alpha


def householder_qr(C: np.ndarray):
    """Thin QR, C = Q R, Q (m x l) orthonormal, R (l x l) upper triangular
    with diag(R) >= 0 (Sec. III: C1 = Q1 R1, C2 = Q2 R2; the paper fixes no
    sign, diag(R) >= 0 makes Q unique for full-rank C).

    Column j: reflector from R[j:, j], applied to the trailing columns; Q is
    formed by applying the reflectors, last first, to the first l columns of I.
    A rank-deficient C still yields an orthonormal Q (its extra columns are
    an arbitrary orthonormal completion).
    """
    R = np.array(C, dtype=np.float64, copy=True)
    m, l = R.shape
    if l > m:
        raise ValueError("householder_qr needs m >= l")
    vs, betas = [], []
    for j in range(l):
        v, beta, alpha = house(R[j:, j])
        if beta != 0.0:
            w = v @ R[j:, j:]
            R[j:, j:] -= beta * np.outer(v, w)
        R[j, j] = alpha
        R[j + 1:, j] = 0.0
        vs.append(v)
        betas.append(beta)
    Q = np.zeros((m, l))
    Q[:l, :l] = np.eye(l)
    for j in range(l - 1, -1, -1):
        v, beta = vs[j], betas[j]
        if beta != 0.0:
            w = v @ Q[j:, j:]
            Q[j:, j:] -= beta * np.outer(v, w)
    R = np.triu(R[:l, :l])
    d = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return Q * d[None, :], R * d[:, None]


# ============================================================================ QRCP
def qrcp(D: np.ndarray):
    """Householder QR with Businger-Golub column pivoting of a square block:
    D P = Q R, i.e. D = Q R P^T (Sec. III, Eq. (D = Q~ R~ P~^T); Alg. 2 step 6).

    Step j brings in the remaining column whose trailing part (rows j:) has
    the largest 2-norm; the norms are recomputed exactly at every step and
    ties go to the lowest column index.  diag(R) >= 0 afterwards (rows of R
    and columns of Q flipped together).  Returns Q, R, perm with
    (D P)[:, j] = D[:, perm[j]].
    """
    R = np.array(D, dtype=np.float64, copy=True)
    n = R.shape[0]
    if R.shape[1] != n:
        raise ValueError("qrcp expects a square core")
    perm = np.arange(n)
    vs, betas = [], []
    for j in range(n):
        norms = np.einsum("ij,ij->j", R[j:, j:], R[j:, j:])
        p = j + int(np.argmax(norms))            # first maximum: lowest index wins ties
        if p != j:
            R[:, [j, p]] = R[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        v, beta, alpha = house(R[j:, j])
        if beta != 0.0:
            w = v @ R[j:, j:]
            R[j:, j:] -= beta * np.outer(v, w)
        R[j, j] = alpha
        R[j + 1:, j] = 0.0
        vs.append(v)
        betas.append(beta)
    Q = np.eye(n)
    for j in range(n - 1, -1, -1):
        v, beta = vs[j], betas[j]
        if beta != 0.0:
            w = v @ Q[j:, j:]
            Q[j:, j:] -= beta * np.outer(v, w)
    R = np.triu(R)
    d = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return Q * d[None, :], R * d[:, None], perm


def qlp(D: np.ndarray):
    """Pivoted QLP of the core (Stewart's QLP approximation of the SVD, SIAM J. Sci.
    Comput. 20 (1999): a QRCP followed by an unpivoted QR of R^T), the alternative
    to Eq. (D = Q~ R~ P~^T) for the l x l core:
        D P = Q R,  R^T = Qh Rh   =>   D = Q L W^T,  L = Rh^T lower triangular, W = P Qh.
    Returns Q, L, W, perm (the QRCP's) and Qh; diag(L) >= 0.
    """
    Q, R, perm = qrcp(D)
    Qh, Rh = householder_qr(R.T)
    n = R.shape[0]
    P = np.zeros((n, n))
    P[perm, np.arange(n)] = 1.0                  # (D P)[:, j] = D[:, perm[j]]
    return Q, Rh.T.copy(), gemm(P, Qh), perm, Qh


# ============================================================================ Jacobi SVD
def _round_robin(n: int):
    """Rounds of disjoint pairs covering every pair once (circle method), n even."""
    players = list(range(n))
    rounds = []
    for _ in range(n - 1):
        half = n // 2
        rounds.append((np.array(players[:half]), np.array(players[half:][::-1])))
        players = [players[0]] + [players[-1]] + players[1:-1]
    return rounds


def jacobi_svd(M: np.ndarray, vectors: bool = False, tol: float = 1e-15, max_sweeps: int = 80):
    """One-sided cyclic Jacobi (Hestenes) SVD in float64 (Sec. II, Eq. (SVD)).

    Columns p, q with alpha = |a_p|^2, beta = |a_q|^2, gamma = a_p.a_q are
    rotated by the angle that zeroes gamma:
        zeta = (beta - alpha) / (2 gamma),  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
        c = 1/sqrt(1 + t^2),  s = c t,  a_p <- c a_p - s a_q,  a_q <- s a_p + c a_q,
    sweeping all pairs (disjoint pairs rotated together) until every pair has
    |gamma| <= tol sqrt(alpha beta).  Singular values are the final column norms,
    returned in non-increasing order.  A brute-force tool for small inputs.
    """
    M = np.asarray(M, dtype=np.float64)
    trans = M.shape[0] < M.shape[1]
    A = (M.T if trans else M).copy()
    m, n = A.shape
    pad = n % 2
    if pad:
        A = np.hstack([A, np.zeros((m, 1))])
    N = A.shape[1]
    V = np.eye(N)
    rounds = _round_robin(N)
    for _ in range(max_sweeps):
        rotated = False
        for P, Qi in rounds:
            ap, aq = A[:, P], A[:, Qi]
            alpha = np.einsum("ij,ij->j", ap, ap)
            beta = np.einsum("ij,ij->j", aq, aq)
            gamma = np.einsum("ij,ij->j", ap, aq)
            act = np.abs(gamma) > tol * np.sqrt(alpha * beta)
            act &= (alpha > 0) & (beta > 0)
            if not act.any():
                continue
            rotated = True
            g = np.where(act, gamma, 1.0)
            zeta = (beta - alpha) / (2.0 * g)
            sgn = np.where(zeta >= 0.0, 1.0, -1.0)
            t = sgn / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
            t = np.where(act, t, 0.0)
            c = 1.0 / np.sqrt(1.0 + t * t)
            s = c * t
            A[:, P], A[:, Qi] = c * ap - s * aq, s * ap + c * aq
            vp, vq = V[:, P], V[:, Qi]
            V[:, P], V[:, Qi] = c * vp - s * vq, s * vp + c * vq
        if not rotated:
            break
    sv = np.sqrt(np.einsum("ij,ij->j", A, A))
    order = np.argsort(-sv, kind="stable")[:n]
    sv = sv[order]
    if not vectors:
        return sv
    V = V[:n, order]
    U = np.zeros((m, n))
    nz = sv > 0
    U[:, nz] = A[:, order][:, nz] / sv[nz][None, :]
    if trans:
        return V, sv, U          # M = V diag(sv) U^T  ->  left vectors are V
    return U, sv, V


def pinv(M: np.ndarray) -> np.ndarray:
    """Moore-Penrose pseudo-inverse from the Jacobi SVD, cutoff l*eps*sigma_max."""
    U, s, V = jacobi_svd(M, vectors=True)
    cut = max(M.shape) * EPS64 * (s[0] if len(s) else 0.0)
    inv = np.where(s > cut, 1.0 / np.where(s > cut, s, 1.0), 0.0)
    return (V * inv[None, :]) @ U.T


# ============================================================================ CoR-UTV
def _check(m, n, k, l, q):
    if not (1 <= k <= l):
        raise ValueError("need 1 <= k <= l")
    if not (l < min(m, n)):
        raise ValueError("need l < min(m, n)")
    if q < 0:
        raise ValueError("need q >= 0")


def corutv(A: np.ndarray, Phi: np.ndarray, k: int, l: int, q: int = 0,
           core: str = "exact", orth: str = "stabilised", side: str = "right", A_core=None,
           factor: str = "qrcp") -> dict:
    """CoR-UTV (Alg. 2 for q = 0, Alg. 3 for q >= 0) in float64.

    side="right": the paper's order, Phi (= Psi) is n x l and C1 = A Psi first;
    returns A ~ U T V^T with T upper triangular.
    side="left":  the m < n modification of Sec. III, i.e. the same algorithm
    run on A^T with Phi m x l (sketch A^T Phi first); returns the ULV form
    A ~ U T V^T with T lower triangular.

    orth="stabilised": orthonormalise C1 and C2 at every power step (range
    finding with the same final Q1, Q2 as the literal loop in exact
    arithmetic); orth="literal": Alg. 3 as printed (products only, one QR of
    each sketch at the end).

    core="exact": D = Q1^T A Q2 (Sec. III, Eq. (D)); core="approx":
    D_approx = Q1^T C1 (Q2^T C2_prev)^+ (Eq. (D_approx)), C2_prev being the
    non-updated sketch that produced the last C1.

    factor="qrcp": the core's rank-revealing factorisation is the QRCP of
    Eq. (D = Q~ R~ P~^T), T = R~ upper triangular; factor="qlp": its QLP
    (see qlp), T = L lower triangular and V = Q2 P~ Qh (the URV becomes a ULV;
    the diagonal of L tracks the singular values more closely).

    A_core (optional, same shape as A, core="exact" only): the correction
    pass of a low-precision A -- the range finding runs on A, the core is
    the projection D = Q1^T A_core Q2 (Eq. (D)) of the full-precision matrix
    onto the bases found.

    Returns U, T, V, perm (V[:, j] = Q2[:, perm[j]] for side="right"; for
    side="left" the permutation acts on U), plus the intermediates.
    """
    A = np.asarray(A, dtype=np.float64)
    Phi = np.asarray(Phi, dtype=np.float64)
    if A_core is not None:
        A_core = np.asarray(A_core, dtype=np.float64)
        if A_core.shape != A.shape or core != "exact":
            raise ValueError("A_core must match A and needs core='exact'")
    if side == "left":
        r = corutv(A.T, Phi, k, l, q, core=core, orth=orth, side="right",
                   A_core=None if A_core is None else A_core.T, factor=factor)
        out = dict(r)
        out["U"], out["V"] = r["V"], r["U"]
        out["T"] = r["T"].T.copy()
        out["side"] = "left"
        return out
    m, n = A.shape
    _check(m, n, k, l, q)
    if Phi.shape != (n, l):
        raise ValueError(f"Phi must be {n} x {l}")

    if orth == "stabilised":
        X = Phi
        for _ in range(q + 1):
            C1 = gemm(A, X)                      # Alg. 3 step 3
            Q1, R1 = householder_qr(C1)
            C2 = gemm(A.T, Q1)                   # Alg. 3 step 4 (on the orthonormalised sketch)
            Q2, R2 = householder_qr(C2)
            X_prev, X = X, Q2
    elif orth == "literal":
        C2 = Phi
        for _ in range(q + 1):
            X_prev = C2
            C1 = gemm(A, C2)                     # Alg. 3 step 3
            C2 = gemm(A.T, C1)                   # Alg. 3 step 4
        Q1, R1 = householder_qr(C1)              # Alg. 3 step 6
        Q2, R2 = householder_qr(C2)
    else:
        raise ValueError("orth must be 'stabilised' or 'literal'")

    if core == "exact":
        D = gemm(Q1.T, gemm(A if A_core is None else A_core, Q2))   # Alg. 2 step 5
    elif core == "approx":
        D = gemm(gemm(Q1.T, C1), pinv(gemm(Q2.T, X_prev)))   # Eq. (D_approx)
    else:
        raise ValueError("core must be 'exact' or 'approx'")

    if factor == "qrcp":
        Qt, Rt, perm = qrcp(D)                   # Alg. 2 step 6
        T = Rt
        V = Q2[:, perm]                          # V = Q2 P~ (columns of Q2 in pivot order)
    elif factor == "qlp":
        Qt, T, _, perm, Qh = qlp(D)
        V = gemm(Q2[:, perm], Qh)                # V = Q2 P~ Qh
    else:
        raise ValueError("factor must be 'qrcp' or 'qlp'")
    U = gemm(Q1, Qt)                             # Alg. 2 step 7
    return dict(U=U, T=T, V=V, perm=perm, D=D, Q1=Q1, Q2=Q2, R1=R1, R2=R2,
                C1=C1, Qt=Qt, side="right")


def rank_k(U: np.ndarray, T: np.ndarray, V: np.ndarray, k: int) -> np.ndarray:
    """Rank-k view U(:,1:k) T(1:k,:) V^T (Sec. VI-B2, Eq. (CoR rank-k))."""
    return gemm(gemm(U[:, :k], T[:k, :]), V.T)


# ============================================================================ quality tools
def fro_residual(A, U, T, V, k: int | None = None) -> float:
    """||A - U T V^T||_F (or of the rank-k view), formed explicitly."""
    B = rank_k(U, T, V, k) if k is not None else gemm(gemm(U, T), V.T)
    return float(np.linalg.norm(np.asarray(A, dtype=np.float64) - B))


def spectral_residual(A, U, T, V, k: int | None = None, iters: int = 50, seed: int = 7, x0=None) -> float:
    """||A - U T V^T||_2 (or of the rank-k view) estimated by power iteration on
    R^T R (R applied as an operator, never formed): per step y = R x,
    x = R^T y / ||R^T y||; the estimate is ||R x|| for the final x.  The start
    vector is x0 if given, else a seeded Gaussian draw; either is normalised."""
    A = np.asarray(A, dtype=np.float64)
    kk = T.shape[0] if k is None else k
    Uk, Tk = U[:, :kk], T[:kk, :]

    def rv(x):
        return A @ x - Uk @ (Tk @ (V.T @ x))

    def rtv(y):
        return A.T @ y - V @ (Tk.T @ (Uk.T @ y))

    if x0 is None:
        x = np.random.default_rng(seed).standard_normal(A.shape[1])
    else:
        x = np.array(x0, dtype=np.float64)
    x /= np.linalg.norm(x)
    s = 0.0
    for _ in range(iters):
        y = rv(x)
        s = np.linalg.norm(y)
        x = rtv(y)
        nx = np.linalg.norm(x)
        if nx == 0.0:
            return 0.0
        x /= nx
    return float(np.linalg.norm(rv(x)))


def factor_distance(U1, T1, V1, U2, T2, V2) -> float:
    """rho = ||U1 T1 V1^T - U2 T2 V2^T||_F / ||U2 T2 V2^T||_F, computed in a
    joint orthonormal basis so that small differences do not cancel:
    with Qu = orth([U1 U2]), Qv = orth([V1 V2]) the difference is
    Qu (Qu^T U1 T1 V1^T Qv - Qu^T U2 T2 V2^T Qv) Qv^T.
    When 2l exceeds a dimension the products are formed explicitly."""
    l1, l2 = U1.shape[1], U2.shape[1]
    if U1.shape[0] < l1 + l2 or V1.shape[0] < l1 + l2:
        X1 = gemm(gemm(U1, T1), V1.T)
        X2 = gemm(gemm(U2, T2), V2.T)
        return float(np.linalg.norm(X1 - X2) / np.linalg.norm(X2))
    Qu, _ = householder_qr(np.hstack([U1, U2]))
    Qv, _ = householder_qr(np.hstack([V1, V2]))
    X1 = gemm(gemm(gemm(Qu.T, U1), T1), gemm(V1.T, Qv))
    X2 = gemm(gemm(gemm(Qu.T, U2), T2), gemm(V2.T, Qv))
    return float(np.linalg.norm(X1 - X2) / np.linalg.norm(X2))


def orthonormality_error(Q: np.ndarray) -> float:
    """max |Q^T Q - I|."""
    G = gemm(Q.T, Q)
    return float(np.abs(G - np.eye(G.shape[0])).max())
