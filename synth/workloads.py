"""Seeded synthetic workloads (test and benchmark inputs only).

Shapes, spectra and structure follow the paper's test matrices (Sec. VI-A:
NoisyLowRank-I/II and the fast-decay matrix; Sec. VI-C synthetic robust-PCA
data) and the five benchmark configurations of this library.  All random
values come from `synth.counter` (SplitMix64 + Box-Muller), so any slice of
any input can be regenerated without the rest.

Seeds: A (and its factors) 1000+c, Phi 2000+c, noise 3000+c,
arrivals/mixes 4000+c, extra trials +100*t.

This module holds no arithmetic of the factorisation method: it builds
inputs (products of generated factors, a library QR to draw Haar-orthonormal
factors, scaling by a library 2-norm) and nothing else.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import counter as C


# ----------------------------------------------------------------------- spectra
def sigma_config1(n: int, k: int = 20, exact_rank: bool = False) -> np.ndarray:
    """sigma_i = 1 for i <= k, 1e-3/(i-k) after (0 after k if exact_rank)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    s = np.where(i <= k, 1.0, 1e-3 / np.maximum(i - k, 1.0))
    if exact_rank:
        s[k:] = 0.0
    return s


def sigma_power(r: int, p: float = 1.5) -> np.ndarray:
    """sigma_i = i^-p, i = 1..r (the 20000x20000 single-solve workload)."""
    return np.arange(1, r + 1, dtype=np.float64) ** (-p)


def sigma_exp(r: int, t: float = 30.0) -> np.ndarray:
    """sigma_i = exp(-i/t), i = 1..r (the 32768x16384 mixed-precision workload)."""
    return np.exp(-np.arange(1, r + 1, dtype=np.float64) / t)


def sigma_noisy_lowrank(order: int, k: int) -> np.ndarray:
    """Sec. VI-A Matrix 1: linear decay from 1 to 1e-9 over the whole order,
    zero after the numerical rank k (the reading that reproduces Fig. 1's SVD
    curve: sigma_20 = 0.98098 before noise)."""
    s = np.linspace(1.0, 1e-9, order)
    s[k:] = 0.0
    return s


def sigma_fast_decay(order: int, k: int = 10) -> np.ndarray:
    """Sec. VI-A Matrix 2: 1 for j <= k, (j-k+1)^-2 after."""
    j = np.arange(1, order + 1, dtype=np.float64)
    return np.where(j <= k, 1.0, (j - k + 1.0) ** -2)


# ----------------------------------------------------------------------- pieces
def gaussian(seed: int, rows: int, cols: int) -> np.ndarray:
    return C.normal_block_np(seed, cols, 0, rows, 0, cols)


def haar_orthonormal(seed: int, rows: int, cols: int) -> np.ndarray:
    """Q factor (sign-fixed, so Haar distributed) of a seeded Gaussian matrix.
    LAPACK's QR (numpy) is used only to draw the test matrix."""
    g = gaussian(seed, rows, cols)
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def phi(n: int, l: int, c: int = 1, trial: int = 0) -> np.ndarray:
    """Gaussian test matrix Psi (n x l), seed 2000+c (+100*trial)."""
    return gaussian(C.stream_seed(2000 + c + 100 * trial), n, l)


def phi_t(n: int, l: int, c: int = 1, trial: int = 0, device="cpu"):
    """Torch twin of phi(), generated on `device` (float64)."""
    return C.normal_block_t(C.stream_seed(2000 + c + 100 * trial), l, 0, n, 0, l, device=device)


# ----------------------------------------------------------------------- config 1
@dataclass
class Dense:
    A: np.ndarray
    sigma: np.ndarray            # singular values of the noise-free part
    k: int
    l: int
    q: int
    meta: dict = field(default_factory=dict)


def config1(c: int = 1, exact_rank: bool = False, noise_std: float = 1e-6,
            m: int = 2000, n: int = 1500, k: int = 20, l: int = 30, q: int = 0) -> Dense:
    """Plain FP64 solve: A = U0 diag(sigma) V0^T + N(0, noise_std^2) noise,
    U0 (m x n), V0 (n x n) Haar-orthonormal.  noise_std is the standard
    deviation (the reading of "N(0, 1e-6)")."""
    base = 1000 + c
    U0 = haar_orthonormal(C.stream_seed(base, 0), m, n)
    V0 = haar_orthonormal(C.stream_seed(base, 1), n, n)
    s = sigma_config1(n, k, exact_rank)
    A = (U0 * s[None, :]) @ V0.T
    if noise_std and not exact_rank:
        A = A + noise_std * gaussian(C.stream_seed(3000 + c), m, n)
    return Dense(A, s, k, l, q, {"U0": U0, "V0": V0, "noise_std": 0.0 if exact_rank else noise_std})


# ----------------------------------------------------------------------- Sec. VI-A
def noisy_lowrank(order: int = 1000, k: int = 20, gap: float = 0.01, c: int = 1) -> Dense:
    """NoisyLowRank-I (gap 0.01) / -II (gap 0.1): A = U diag(sigma) V^T + E,
    E Gaussian scaled so that ||E||_2 = gap * sigma_k."""
    base = 1000 + c
    U = haar_orthonormal(C.stream_seed(base, 10), order, order)
    V = haar_orthonormal(C.stream_seed(base, 11), order, order)
    s = sigma_noisy_lowrank(order, k)
    E = gaussian(C.stream_seed(3000 + c, 10), order, order)
    E *= gap * s[k - 1] / np.linalg.norm(E, 2)
    A = (U * s[None, :]) @ V.T + E
    return Dense(A, s, k, 2 * k, 0, {"gap": gap})


def fast_decay(order: int = 1000, k: int = 10, c: int = 1) -> Dense:
    base = 1000 + c
    U = haar_orthonormal(C.stream_seed(base, 20), order, order)
    V = haar_orthonormal(C.stream_seed(base, 21), order, order)
    s = sigma_fast_decay(order, k)
    return Dense((U * s[None, :]) @ V.T, s, k, 2 * k, 0, {})


# ----------------------------------------------------------------------- configs 2/3
@dataclass
class GaussLowRank:
    """A = G1 diag(sigma) G2^T + noise_std * N, G1 (m x r), G2 (n x r) Gaussian/sqrt(r).
    Element (i, j) of the noise is normal(seed_noise, i*n + j), so any block of A
    can be regenerated on its own."""
    m: int
    n: int
    sigma: np.ndarray
    noise_std: float
    c: int

    @property
    def r(self) -> int:
        return len(self.sigma)

    def seeds(self):
        base = 1000 + self.c
        return C.stream_seed(base, 30), C.stream_seed(base, 31), C.stream_seed(3000 + self.c, 30)

    def g1(self, r0: int, r1: int) -> np.ndarray:
        s1, _, _ = self.seeds()
        return C.normal_block_np(s1, self.r, r0, r1, 0, self.r) / np.sqrt(self.r)

    def g2(self, c0: int, c1: int) -> np.ndarray:
        _, s2, _ = self.seeds()
        return C.normal_block_np(s2, self.r, c0, c1, 0, self.r) / np.sqrt(self.r)

    def block(self, r0: int, r1: int, c0: int, c1: int) -> np.ndarray:
        """A[r0:r1, c0:c1] in float64 (numpy)."""
        _, _, sn = self.seeds()
        out = (self.g1(r0, r1) * self.sigma[None, :]) @ self.g2(c0, c1).T
        if self.noise_std:
            out += self.noise_std * C.normal_block_np(sn, self.n, r0, r1, c0, c1)
        return out

    def block_t(self, r0: int, r1: int, c0: int, c1: int, device="cpu", dtype=None, chunk: int = 2048):
        """A[r0:r1, c0:c1] generated with torch on `device`, cast to `dtype`
        (float64 arithmetic, row chunks of `chunk`)."""
        import torch
        dtype = dtype or torch.float64
        s1, s2, sn = self.seeds()
        sig = torch.as_tensor(self.sigma, dtype=torch.float64, device=device)
        g2 = C.normal_block_t(s2, self.r, c0, c1, 0, self.r, device=device) / np.sqrt(self.r)
        g2s = (g2 * sig[None, :]).T.contiguous()
        out = torch.empty((r1 - r0, c1 - c0), dtype=dtype, device=device)
        for a in range(r0, r1, chunk):
            b = min(r1, a + chunk)
            g1 = C.normal_block_t(s1, self.r, a, b, 0, self.r, device=device) / np.sqrt(self.r)
            blk = g1 @ g2s
            if self.noise_std:
                blk += self.noise_std * C.normal_block_t(sn, self.n, a, b, c0, c1, device=device)
            out[a - r0:b - r0] = blk.to(dtype)
        return out


def config2(c: int = 2, m: int = 20000, n: int = 20000) -> GaussLowRank:
    """Large FP32 single solve: sigma_i = i^-1.5 (i <= 400), noise std 1e-8."""
    return GaussLowRank(m, n, sigma_power(400), 1e-8, c)


def config3(c: int = 3, m: int = 32768, n: int = 16384) -> GaussLowRank:
    """Mixed-precision workload: sigma_i = exp(-i/30) (i <= 400), noise std 1e-8."""
    return GaussLowRank(m, n, sigma_exp(400), 1e-8, c)


# ----------------------------------------------------------------------- config 4 / RPCA
@dataclass
class LowRankSparse:
    """L = X Y^T (X m x r, Y n x r standard Gaussian) plus a sparse part:
    each entry is, with probability `density`, shifted by U[-amp, amp]."""
    m: int
    n: int
    r: int
    density: float
    amp: float
    seed: int

    def dense(self) -> np.ndarray:
        sx, sy, sb, sv = (C.stream_seed(self.seed, i) for i in range(4))
        X = C.normal_block_np(sx, self.r, 0, self.m, 0, self.r)
        Y = C.normal_block_np(sy, self.r, 0, self.n, 0, self.r)
        A = X @ Y.T
        hit = C.uniform_block_np(sb, self.n, 0, self.m, 0, self.n) < self.density
        val = (2.0 * C.uniform_block_np(sv, self.n, 0, self.m, 0, self.n) - 1.0) * self.amp
        return A + np.where(hit, val, 0.0)

    def dense_t(self, device="cpu", dtype=None):
        import torch
        dtype = dtype or torch.float64
        sx, sy, sb, sv = (C.stream_seed(self.seed, i) for i in range(4))
        X = C.normal_block_t(sx, self.r, 0, self.m, 0, self.r, device=device)
        Y = C.normal_block_t(sy, self.r, 0, self.n, 0, self.r, device=device)
        A = X @ Y.T
        hit = C.uniform_block_t(sb, self.n, 0, self.m, 0, self.n, device=device) < self.density
        val = (2.0 * C.uniform_block_t(sv, self.n, 0, self.m, 0, self.n, device=device) - 1.0) * self.amp
        return (A + torch.where(hit, val, torch.zeros_like(val))).to(dtype)


def _uniform_int(seed: int, i: int, lo: int, hi: int) -> int:
    u = float(C.uniform_np(seed, np.array([i], dtype=np.uint64))[0])
    return lo + min(int(u * (hi - lo + 1)), hi - lo)


@dataclass
class Problem:
    m: int
    n: int
    r: int
    l: int
    q: int
    k: int
    content: LowRankSparse
    phi_seed: int


def batch_config4(count: int = 1024, c: int = 4) -> list[Problem]:
    """Batched uneven solves: m ~ U{256..4096}, n ~ U{128..2048}, r ~ U{4..32},
    l = r + 8, q = 1, 5% sparse entries U[-10, 10]."""
    s = C.stream_seed(4000 + c, 0)
    probs = []
    for p in range(count):
        m = _uniform_int(s, 3 * p + 0, 256, 4096)
        n = _uniform_int(s, 3 * p + 1, 128, 2048)
        r = _uniform_int(s, 3 * p + 2, 4, 32)
        probs.append(Problem(m, n, r, r + 8, 1, r,
                             LowRankSparse(m, n, r, 0.05, 10.0, C.stream_seed(1000 + c, 1000 + p)),
                             C.stream_seed(2000 + c, 1000 + p)))
    return probs


def problem_phi(p: Problem, rows: int) -> np.ndarray:
    return C.normal_block_np(p.phi_seed, p.l, 0, rows, 0, p.l)


def problem_phi_t(p: Problem, rows: int, device="cpu"):
    return C.normal_block_t(p.phi_seed, p.l, 0, rows, 0, p.l, device=device)


def rpca_synthetic(n: int, rank_frac: float = 0.05, sparse_frac: float = 0.05, c: int = 6):
    """Sec. VI-C synthetic robust-PCA data: L = U V^T (rank r = rank_frac*n,
    Gaussian factors), S with sparse_frac*n^2 entries of value +-80 at random
    positions.  Returns (M, L, S)."""
    r = max(1, int(round(rank_frac * n)))
    base = 1000 + c
    U = C.normal_block_np(C.stream_seed(base, 40), r, 0, n, 0, r)
    V = C.normal_block_np(C.stream_seed(base, 41), r, 0, n, 0, r)
    L = U @ V.T
    u = C.uniform_block_np(C.stream_seed(base, 42), n, 0, n, 0, n)
    sgn = np.where(C.uniform_block_np(C.stream_seed(base, 43), n, 0, n, 0, n) < 0.5, -80.0, 80.0)
    S = np.where(u < sparse_frac, sgn, 0.0)
    return L + S, L, S


# ----------------------------------------------------------------------- config 5
@dataclass
class Request:
    t_arrive: float
    m: int
    n: int
    k: int
    l: int
    q: int
    content: LowRankSparse
    phi_seed: int


SERVING_SIZES = ((1024, 512), (8192, 2048), (76800, 200))
SERVING_MIX = (0.70, 0.25, 0.05)


def serving_stream(rate: float = 2000.0, duration: float = 60.0, c: int = 5,
                   start: int = 0) -> list[Request]:
    """Poisson arrivals at `rate` req/s over `duration` s; sizes drawn 70/25/5%
    from 1024x512, 8192x2048, 76800x200 (pixels x frames); rank-5 content plus
    5% sparse outliers; k ~ U{5,20,50}, l = k + 10, q ~ U{0,1}."""
    s = C.stream_seed(4000 + c, 1)
    t = 0.0
    out = []
    i = start
    while True:
        u = float(C.uniform_np(s, np.array([5 * i], dtype=np.uint64))[0])
        t += -np.log1p(-u) / rate
        if t > duration:
            break
        us = float(C.uniform_np(s, np.array([5 * i + 1], dtype=np.uint64))[0])
        cls = 0 if us < SERVING_MIX[0] else (1 if us < SERVING_MIX[0] + SERVING_MIX[1] else 2)
        m, n = SERVING_SIZES[cls]
        k = (5, 20, 50)[_uniform_int(s, 5 * i + 2, 0, 2)]
        q = _uniform_int(s, 5 * i + 3, 0, 1)
        out.append(Request(t, m, n, k, k + 10, q,
                           LowRankSparse(m, n, 5, 0.05, 10.0, C.stream_seed(1000 + c, 10 + i)),
                           C.stream_seed(2000 + c, 10 + i)))
        i += 1
    return out
