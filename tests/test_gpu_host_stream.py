"""GPU parity of corutv_solve_host: A stays in host memory and every pass streams
it through the device ring in row chunks (the externally stored matrix of
Sec. I, read 2q + 3 times, Sec. IV-C).  The factors are compared with the FP64
oracle on the same inputs at the tolerances of the resident solve (the chunked
passes differ from the resident ones only in the order of FP sums), over chunk
sizes that give one chunk, a ragged last chunk and more chunks than ring
buffers; ||A||_F^2 is summed over the chunks of the first pass, so the host
matrix is read exactly 2q + 3 times.
"""
import numpy as np
import pytest

from oracle import corutv_oracle as O
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1810_07323_gb300 import corutv

TOL = {"f64": 1e-10, "simt": 1e-4, "tf32": 1e-3}


def _host(A, dt, pinned=True, pad=0):
    """Host copy of A in dtype dt, page-locked on request, row pitch n + pad."""
    m, n = A.shape
    buf = torch.empty((m, n + pad), dtype=dt, pin_memory=pinned)
    Ah = buf[:, :n]
    Ah.copy_(torch.tensor(A, dtype=torch.float64).to(dt))
    return Ah


def _np(r):
    return r.U.double().cpu().numpy(), r.T.cpu().numpy(), r.V.double().cpu().numpy(), r.perm.cpu().numpy()


def _structure(U, T, V, perm, l, side="right", orth_tol=1e-12):
    tri = np.tril(T, -1) if side == "right" else np.triu(T, 1)
    assert np.abs(tri).max() == 0.0
    d = np.diag(T)
    assert np.all(d >= 0) and np.all(np.diff(d) <= 1e-12 * max(d[0], 1e-300))
    assert sorted(perm) == list(range(l))
    assert O.orthonormality_error(U) < orth_tol
    assert O.orthonormality_error(V) < orth_tol


@pytest.fixture(scope="module")
def slice2():
    """4000 x 3000 slice of the 20000 x 20000 workload (sigma_i = i^-1.5)."""
    g = W.config2()
    return g.block(0, 4000, 0, 3000), W.phi(20000, 120)[:3000], W.phi(20000, 120)[:4000]


@pytest.mark.parametrize("chunk", [0, 512, 1152])
@pytest.mark.parametrize("mma", ["tf32", "simt"])
def test_fp32_streamed_parity(slice2, chunk, mma):
    A, phi_r, _ = slice2
    Ah = _host(A, torch.float32, pad=5)
    P = torch.tensor(phi_r, dtype=torch.float32, device="cuda")
    r = corutv.solve_host(Ah, P, 100, 120, 1, mma=mma, want_fro2=True, chunk_rows=chunk)
    assert r.info.status == 0
    U, T, V, perm = _np(r)
    A64 = Ah.double().numpy()
    ref = O.corutv(A64, P.double().cpu().numpy(), 100, 120, 1)
    rho = O.factor_distance(U, T, V, ref["U"], ref["T"], ref["V"])
    assert rho < TOL[mma], rho
    _structure(U, T, V, perm, 120, orth_tol=2e-5)
    a2 = np.sum(A64 ** 2)
    assert abs(r.info.fro2_A - a2) < 1e-6 * a2
    assert r.info.passes_over_A == 5            # 2q + 3: ||A||^2 rides on the first pass


def test_fp32_streamed_matches_resident(slice2):
    """Same engine, same inputs: the streamed solve and the resident one agree to FP32
    summation-order level (the TF32 products round the same elements)."""
    A, phi_r, _ = slice2
    Ah = _host(A, torch.float32)
    P = torch.tensor(phi_r, dtype=torch.float32, device="cuda")
    rs = corutv.solve_host(Ah, P, 100, 120, 0, mma="simt", chunk_rows=384)
    rd = corutv.solve(Ah.cuda(), P, 100, 120, 0, mma="simt")
    Us, Ts, Vs, _ = _np(rs)
    Ud, Td, Vd, _ = _np(rd)
    assert O.factor_distance(Us, Ts, Vs, Ud, Td, Vd) < 1e-5


def test_fp32_streamed_left_ragged(slice2):
    """LEFT (ULV): the first product is A^T Psi, summed over 32 chunks of 128 rows
    (4000 = 31 x 128 + 32: a ragged last chunk), from pageable memory."""
    A, _, phi_l = slice2
    Ah = _host(A, torch.float32, pinned=False)
    P = torch.tensor(phi_l, dtype=torch.float32, device="cuda")
    r = corutv.solve_host(Ah, P, 100, 120, 1, side="left", mma="simt", chunk_rows=128)
    U, T, V, perm = _np(r)
    ref = O.corutv(Ah.double().numpy(), P.double().cpu().numpy(), 100, 120, 1, side="left")
    assert O.factor_distance(U, T, V, ref["U"], ref["T"], ref["V"]) < TOL["simt"]
    _structure(U, T, V, perm, 120, side="left", orth_tol=2e-5)


@pytest.mark.parametrize("core", ["exact", "sketch"])
def test_fp64_streamed_parity(core):
    d = W.config1()
    Ah = _host(d.A, torch.float64, pad=3)
    phi = W.phi(1500, 30)
    P = torch.tensor(phi, dtype=torch.float64, device="cuda")
    r = corutv.solve_host(Ah, P, 20, 30, 2, core=core, want_fro2=True, chunk_rows=256)
    U, T, V, perm = _np(r)
    ref = O.corutv(d.A, phi, 20, 30, 2)          # core = SKETCH forms the same D from the saved C2
    assert O.factor_distance(U, T, V, ref["U"], ref["T"], ref["V"]) < TOL["f64"]
    assert np.array_equal(perm, ref["perm"])
    _structure(U, T, V, perm, 30)
    a2 = np.sum(d.A ** 2)
    assert abs(r.info.fro2_A - a2) < 1e-12 * a2
    assert r.info.passes_over_A == 2 * 2 + (3 if core == "exact" else 2)


def test_streamed_qlp_and_repeat(slice2):
    """QLP of the core on the streamed path, and the ring reused by a second solve on
    the same handle gives the same factors bit for bit."""
    A, phi_r, _ = slice2
    Ah = _host(A, torch.float32)
    P = torch.tensor(phi_r, dtype=torch.float32, device="cuda")
    h = corutv.Handle()
    r1 = corutv.solve_host(Ah, P, 100, 120, 1, factor="qlp", chunk_rows=640, handle=h)
    a = [t.clone() for t in (r1.U, r1.T, r1.V)]
    r2 = corutv.solve_host(Ah, P, 100, 120, 1, factor="qlp", chunk_rows=640, handle=h)
    for x, y in zip(a, (r2.U, r2.T, r2.V)):
        assert torch.equal(x, y)
    U, T, V, _ = _np(r2)
    assert np.abs(np.triu(T, 1)).max() == 0.0        # QLP: T lower triangular
    ref = O.corutv(Ah.double().numpy(), P.double().cpu().numpy(), 100, 120, 1, factor="qlp")
    assert O.factor_distance(U, T, V, ref["U"], ref["T"], ref["V"]) < TOL["tf32"]
    h.close()


def test_streamed_bad_args(slice2):
    A, phi_r, _ = slice2
    Ah = _host(A[:512, :400], torch.float32)
    P = torch.tensor(phi_r[:400, :40], dtype=torch.float32, device="cuda")
    with pytest.raises(corutv.CorutvError):
        corutv.solve_host(Ah, P, 10, 40, 0, chunk_rows=100)          # not a multiple of 128
    with pytest.raises(corutv.CorutvError):
        corutv.solve_host(Ah.to(torch.bfloat16), P, 10, 40, 0)      # host streaming: F32 / F64 only
    with pytest.raises(TypeError):
        corutv.solve_host(Ah.cuda(), P, 10, 40, 0)                  # A must be on the host


@pytest.mark.parametrize("shape,chunk,side", [((200, 150), 128, "right"), ((129, 300), 128, "left"),
                                               ((700, 90), 256, "right")])
def test_streamed_small_shapes(shape, chunk, side):
    """Edge cases: fewer rows than one chunk plus one row, a chunk of 128 rows with a one-row
    tail, m much larger than n; F64 so the comparison is exact to rounding."""
    m, n = shape
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((m, n)) @ np.diag(0.7 ** np.arange(n)) if m >= n else \
        np.diag(0.7 ** np.arange(m)) @ rng.standard_normal((m, n))
    l = 30
    phi = rng.standard_normal((n if side == "right" else m, l))
    Ah = _host(A, torch.float64, pinned=(m % 2 == 0))
    P = torch.tensor(phi, dtype=torch.float64, device="cuda")
    r = corutv.solve_host(Ah, P, 10, l, 1, side=side, want_fro2=True, chunk_rows=chunk)
    U, T, V, perm = _np(r)
    ref = O.corutv(A, phi, 10, l, 1, side=side)
    assert O.factor_distance(U, T, V, ref["U"], ref["T"], ref["V"]) < TOL["f64"]
    assert np.array_equal(perm, ref["perm"])
    _structure(U, T, V, perm, l, side=side)
    a2 = np.sum(A ** 2)
    assert abs(r.info.fro2_A - a2) < 1e-12 * a2


def test_host_read_time():
    """corutv_host_read_time: a kernel reads page-locked host memory directly; the rate is
    positive and finite; unaligned sizes and memory CUDA does not know as page-locked are
    refused before anything is launched."""
    src = torch.ones(1 << 22, dtype=torch.float32, pin_memory=True)     # 16 MiB
    ms = corutv.host_read_time(src)
    assert 0.0 < ms < 1e4
    with pytest.raises(corutv.CorutvError) as e:
        corutv.host_read_time(src[:3])                                   # 12 bytes: not a multiple of 16
    assert e.value.status == corutv.ERR_ALIGN
    with pytest.raises(corutv.CorutvError) as e:
        corutv.host_read_time(torch.ones(1 << 10, dtype=torch.float32))  # pageable
    assert e.value.status == corutv.ERR_INVALID_ARG
