"""ctypes binding of libcorutv (argument marshalling only).

Every step of the computation runs in the library's CUDA kernels; this module
only checks tensor placement, allocates outputs with torch (device memory
plumbing) and forwards raw pointers, sizes and the current CUDA stream to the
C ABI declared in include/corutv.h.  If the shared library is missing the
import fails: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcorutv.so")

# status codes (include/corutv.h)
OK, ERR_INVALID_ARG, ERR_SHAPE, ERR_ALIGN, ERR_OOM, ERR_CUDA, ERR_TIMEOUT = 0, 1, 2, 3, 4, 5, 6
ERR_CHOL_BREAKDOWN, ERR_BUSY, PENDING, ERR_UNSUPPORTED = 7, 8, 9, 10
SIDE = {"right": 0, "left": 1}
CORE = {"exact": 0, "sketch": 1}
DTYPE = {"f64": 0, "f32": 1, "bf16": 2, "fp8": 3}
ORTH = {"stabilised": 0, "strict": 1, "literal": 2}
MMA = {"auto": 0, "tf32": 1, "tf32x3": 2, "simt": 3, "tf32t": 4, "bf16x2": 5}
DIR = {"ax": 0, "aty": 1}


class CorutvError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} (status {status})")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int32), ("l", ctypes.c_int32),
                ("q", ctypes.c_int32), ("side", ctypes.c_int32), ("core", ctypes.c_int32),
                ("orth", ctypes.c_int32), ("a_dtype", ctypes.c_int32), ("mma", ctypes.c_int32),
                ("want_fro2", ctypes.c_int32), ("factor", ctypes.c_int32), ("small_f64", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("tuned", ctypes.c_int32), ("from_cache", ctypes.c_int32), ("gram_cols", ctypes.c_int32),
                ("split_k", ctypes.c_int32), ("tc_order", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("tuned_ms", ctypes.c_double), ("default_ms", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int32), ("l", ctypes.c_int32),
                ("q", ctypes.c_int32), ("side", ctypes.c_int32), ("core", ctypes.c_int32),
                ("orth", ctypes.c_int32), ("a_dtype", ctypes.c_int32), ("mma", ctypes.c_int32),
                ("want_fro2", ctypes.c_int32), ("fuse_power", ctypes.c_int32),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("a_tile_scales", ctypes.c_void_p),
                ("Phi", ctypes.c_void_p), ("ldphi", ctypes.c_int64), ("U", ctypes.c_void_p),
                ("ldu", ctypes.c_int64), ("T", ctypes.c_void_p), ("ldt", ctypes.c_int64),
                ("V", ctypes.c_void_p), ("ldv", ctypes.c_int64), ("perm", ctypes.c_void_p),
                ("reserved", ctypes.c_int64 * 4)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("passes_over_A", ctypes.c_int32),
                ("chol_fallbacks", ctypes.c_int32), ("hbm_passes_over_A", ctypes.c_int32),
                ("chol_shift_rel", ctypes.c_double), ("fro2_A", ctypes.c_double),
                ("fro2_T", ctypes.c_double), ("fro2_Tk", ctypes.c_double)]


class Trace(ctypes.Structure):
    _fields_ = [("solves", ctypes.c_int32), ("pass_launches", ctypes.c_int32), ("launches", ctypes.c_int64),
                ("pass_ms", ctypes.c_double), ("pass_bytes", ctypes.c_double), ("orth_ms", ctypes.c_double),
                ("core_ms", ctypes.c_double), ("qrcp_ms", ctypes.c_double), ("assembly_ms", ctypes.c_double),
                ("fro2_ms", ctypes.c_double), ("corr_launches", ctypes.c_int32), ("reserved1", ctypes.c_int32),
                ("corr_ms", ctypes.c_double), ("corr_bytes", ctypes.c_double), ("quant_ms", ctypes.c_double),
                ("pass_kernel_launches", ctypes.c_int32), ("reserved2", ctypes.c_int32),
                ("pass_kernel_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class RpcaParams(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int32), ("l", ctypes.c_int32),
                ("q", ctypes.c_int32), ("side", ctypes.c_int32), ("mma", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("lam", ctypes.c_double), ("mu0", ctypes.c_double),
                ("rho", ctypes.c_double), ("mu_bar", ctypes.c_double), ("tol", ctypes.c_double),
                ("reserved", ctypes.c_int32 * 4)]


class RpcaInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("zeta", ctypes.c_double), ("mu", ctypes.c_double)]


_lib = None

# every entry point declared in include/corutv.h
EXPORTS = ("corutv_version", "corutv_status_string", "corutv_create", "corutv_destroy", "corutv_set_stream",
           "corutv_workspace_size", "corutv_set_workspace", "corutv_solve", "corutv_info_wait",
           "corutv_set_tracing", "corutv_trace_read", "corutv_pass", "corutv_orthonormalize", "corutv_gram",
           "corutv_qrcp", "corutv_fro2", "corutv_gram_noalloc", "corutv_solve_corrected", "corutv_quantize",
           "corutv_batch_workspace_size", "corutv_solve_batched", "corutv_batch_info_wait",
           "corutv_server_create", "corutv_server_submit", "corutv_server_poll", "corutv_server_stats",
           "corutv_server_launches", "corutv_server_destroy", "corutv_rpca", "corutv_solve_host",
           "corutv_residual_norm2", "corutv_host_read_time", "corutv_set_autotune", "corutv_batch_tuning_read")


def load() -> ctypes.CDLL:
    """Load libcorutv.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1810_07323_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.corutv_version.restype = ctypes.c_int
    lib.corutv_status_string.restype = ctypes.c_char_p
    lib.corutv_status_string.argtypes = [ctypes.c_int]
    lib.corutv_create.argtypes = [ctypes.POINTER(P), P]
    lib.corutv_destroy.argtypes = [P]
    lib.corutv_set_stream.argtypes = [P, P]
    lib.corutv_workspace_size.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)]
    lib.corutv_set_workspace.argtypes = [P, P, ctypes.c_size_t]
    lib.corutv_solve.argtypes = [P, ctypes.POINTER(Params), P, I64, P, P, I64, P, I64, P, I64, P, I64, P]
    lib.corutv_solve_corrected.argtypes = [P, ctypes.POINTER(Params), P, I64, P, P, I64, P, I64, P, I64, P, I64,
                                           P, I64, P]
    lib.corutv_solve_host.argtypes = [P, ctypes.POINTER(Params), P, I64, I64, P, I64, P, I64, P, I64, P, I64, P]
    lib.corutv_residual_norm2.argtypes = [P, ctypes.c_int, P, I64, I64, I64, P, I64, P, I64, P, I64, ctypes.c_int,
                                          ctypes.c_int, P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.corutv_quantize.argtypes = [P, ctypes.c_int, P, I64, I64, I64, P, I64, P]
    lib.corutv_batch_workspace_size.argtypes = [ctypes.c_int, ctypes.POINTER(Problem), ctypes.POINTER(ctypes.c_size_t)]
    lib.corutv_solve_batched.argtypes = [P, ctypes.c_int, ctypes.POINTER(Problem), ctypes.POINTER(Info)]
    lib.corutv_batch_info_wait.argtypes = [P, ctypes.c_int, ctypes.POINTER(Info)]
    lib.corutv_server_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.c_int]
    lib.corutv_server_submit.argtypes = [P, ctypes.POINTER(Problem), ctypes.POINTER(ctypes.c_uint64)]
    lib.corutv_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(Info)]
    lib.corutv_server_stats.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.corutv_server_launches.argtypes = [P, ctypes.POINTER(I64)]
    lib.corutv_server_destroy.argtypes = [P]
    lib.corutv_info_wait.argtypes = [P, ctypes.POINTER(Info)]
    lib.corutv_pass.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, I64, I64, I64, P, P, I64, I32, P,
                                I64]
    lib.corutv_orthonormalize.argtypes = [P, ctypes.c_int, P, I64, I64, I32, P]
    lib.corutv_gram.argtypes = [P, ctypes.c_int, P, I64, P, I64, I64, I32, P]
    lib.corutv_qrcp.argtypes = [P, ctypes.c_int, P, I64, I32, I32, P, P, P, P]
    lib.corutv_fro2.argtypes = [P, ctypes.c_int, P, I64, I64, I64, P, P]
    lib.corutv_gram_noalloc.argtypes = [P, ctypes.c_int, P, I64, P, I64, I64, I32, P]
    lib.corutv_gram_noalloc.restype = ctypes.c_int
    lib.corutv_rpca.argtypes = [P, ctypes.POINTER(RpcaParams), P, I64, P, I64, P, I64, P, I64, P, I64,
                                ctypes.POINTER(RpcaInfo)]
    lib.corutv_host_read_time.argtypes = [P, P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_float)]
    lib.corutv_set_autotune.argtypes = [P, ctypes.c_int, ctypes.c_char_p]
    lib.corutv_batch_tuning_read.argtypes = [P, ctypes.POINTER(BatchTuning)]
    lib.corutv_set_tracing.argtypes = [P, ctypes.c_int]
    lib.corutv_trace_read.argtypes = [P, ctypes.POINTER(Trace)]
    for name in ("corutv_set_tracing", "corutv_trace_read", "corutv_create", "corutv_destroy", "corutv_set_stream", "corutv_workspace_size",
                 "corutv_set_workspace", "corutv_solve", "corutv_info_wait", "corutv_pass",
                 "corutv_orthonormalize", "corutv_gram", "corutv_qrcp", "corutv_fro2", "corutv_solve_corrected",
                 "corutv_quantize", "corutv_batch_workspace_size", "corutv_solve_batched",
                 "corutv_batch_info_wait", "corutv_server_create", "corutv_server_submit", "corutv_server_poll",
                 "corutv_server_stats", "corutv_server_launches", "corutv_server_destroy", "corutv_rpca",
                 "corutv_solve_host",
                 "corutv_residual_norm2", "corutv_host_read_time", "corutv_set_autotune",
                 "corutv_batch_tuning_read"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().corutv_status_string(int(status)).decode()


def version() -> int:
    return load().corutv_version()


def _check(rc: int, what: str):
    if rc != OK:
        raise CorutvError(rc, what)


# ------------------------------------------------------------------ handles
class Handle:
    """A libcorutv handle bound to one CUDA stream (its own lazily grown workspace)."""

    def __init__(self, stream=None):
        import torch
        self._torch = torch
        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib.corutv_create(ctypes.byref(h), ctypes.c_void_p(stream.cuda_stream)), "corutv_create")
        self.h = h

    def close(self):
        if self.h:
            load().corutv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tracing(self, enable: bool = True):
        _check(load().corutv_set_tracing(self.h, 1 if enable else 0), "corutv_set_tracing")

    def trace_read(self) -> Trace:
        t = Trace()
        _check(load().corutv_trace_read(self.h, ctypes.byref(t)), "corutv_trace_read")
        return t

    def set_workspace(self, tensor):
        """Use a caller-owned device tensor as workspace (None: self-allocate)."""
        ptr = 0 if tensor is None else tensor.data_ptr()
        nbytes = 0 if tensor is None else tensor.numel() * tensor.element_size()
        _check(load().corutv_set_workspace(self.h, ctypes.c_void_p(ptr), nbytes), "corutv_set_workspace")


_handles: dict = {}


def handle_for(stream=None) -> Handle:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    key = (stream.device.index if stream.device.index is not None else torch.cuda.current_device(),
           stream.cuda_stream)
    h = _handles.get(key)
    if h is None:
        h = Handle(stream)
        _handles[key] = h
    return h


# ------------------------------------------------------------------ helpers
def _dt_code(t) -> int:
    import torch
    m = {torch.float64: 0, torch.float32: 1, torch.bfloat16: 2}
    if t.dtype in m:
        return m[t.dtype]
    if t.dtype == getattr(torch, "float8_e4m3fn", None):
        return 3
    raise TypeError(f"unsupported dtype {t.dtype}")


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("libcorutv takes device tensors (no CPU path)")


def _rowmajor_ld(t) -> int:
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a 2-D row-major tensor with unit column stride")
    return t.stride(0)


def ld_for(length: int) -> int:
    """Leading dimension the library uses for skinny-transposed buffers."""
    return max(64, (length + 63) // 64 * 64)


@dataclass
class SolveResult:
    U: object
    T: object
    V: object
    perm: object
    info: Info | None


def workspace_size(m, n, k, l, q=0, side="right", core="exact", a_dtype="f32", mma="auto", factor="qrcp",
                   small_f64=0) -> int:
    p = _params(m, n, k, l, q, side, core, DTYPE[a_dtype], mma, False, "stabilised", factor, small_f64)
    out = ctypes.c_size_t()
    _check(load().corutv_workspace_size(ctypes.byref(p), ctypes.byref(out)), "corutv_workspace_size")
    return out.value


FACTOR = {"qrcp": 0, "qlp": 1}


def _params(m, n, k, l, q, side, core, a_dtype_code, mma, want_fro2, orth, factor="qrcp", small_f64=False) -> Params:
    p = Params()
    p.m, p.n, p.k, p.l, p.q = int(m), int(n), int(k), int(l), int(q)
    p.side, p.core, p.orth = SIDE[side], CORE[core], ORTH[orth]
    p.a_dtype, p.mma, p.want_fro2 = a_dtype_code, MMA[mma], 1 if want_fro2 else 0
    p.factor = FACTOR[factor]
    p.small_f64 = int(small_f64)
    return p


def solve(A, Phi, k: int, l: int, q: int = 0, side: str = "right", core: str = "exact", mma: str = "auto",
          a_tile_scales=None, want_fro2: bool = False, out=None, wait: bool = True, handle: Handle | None = None,
          A_ref=None, orth: str = "stabilised", factor: str = "qrcp", small_f64: bool = False):
    """CoR-UTV of a device matrix A (Alg. 2 / Alg. 3): returns U, T, V, perm.

    A: (m, n) row-major float64 / float32 / bfloat16 / float8_e4m3fn (with
    a_tile_scales); Phi: (n, l) for side="right", (m, l) for side="left",
    float64 if A is float64 else float32.  T is float64.
    A_ref: optional float32 (m, n) matrix for the correction pass of a
    bfloat16 / float8 A (corutv_solve_corrected: the core D from A_ref).
    orth: "stabilised" (one shifted CholeskyQR pass for the sketches of the
    earlier power steps), "strict" (shifted CholeskyQR3 for every sketch) or "literal" (Alg. 3 as
    printed: no orthonormalisation inside the power steps, exact core only).
    factor: "qrcp" (T upper triangular) or "qlp" (T lower triangular, V
    = Q2 P~ Qh; float32-path solves).
    small_f64: float32 / bfloat16 / float8 A with the Gram reductions,
    Cholesky factors, core and QRCP in FP64 (corutv_params.small_f64).
    out: optional (U, T, V, perm) preallocated outputs.  wait=True
    synchronises and returns the device info; wait=False leaves the work
    enqueued on the current stream (info is None).
    """
    import torch
    _need_cuda(A, Phi, a_tile_scales, A_ref)
    h = handle or handle_for()
    m, n = A.shape
    code = _dt_code(A)
    fdt = torch.float64 if code == 0 else torch.float32
    if Phi.dtype != fdt:
        raise TypeError(f"Phi must be {fdt}")
    p = _params(m, n, k, l, q, side, core, code, mma, want_fro2, orth, factor, small_f64)
    if out is None:
        dev = A.device
        U = torch.empty((m, l), dtype=fdt, device=dev)
        T = torch.empty((l, l), dtype=torch.float64, device=dev)
        V = torch.empty((n, l), dtype=fdt, device=dev)
        perm = torch.empty((l,), dtype=torch.int32, device=dev)
    else:
        U, T, V, perm = out
    sc = a_tile_scales.data_ptr() if a_tile_scales is not None else 0
    tail = (ctypes.c_void_p(Phi.data_ptr()), _rowmajor_ld(Phi), ctypes.c_void_p(U.data_ptr()), _rowmajor_ld(U),
            ctypes.c_void_p(T.data_ptr()), _rowmajor_ld(T), ctypes.c_void_p(V.data_ptr()), _rowmajor_ld(V),
            ctypes.c_void_p(perm.data_ptr()))
    if A_ref is None:
        rc = load().corutv_solve(h.h, ctypes.byref(p), ctypes.c_void_p(A.data_ptr()), _rowmajor_ld(A),
                                 ctypes.c_void_p(sc), *tail)
        _check(rc, "corutv_solve")
    else:
        if A_ref.dtype != torch.float32 or tuple(A_ref.shape) != (m, n):
            raise TypeError("A_ref must be a float32 (m, n) matrix")
        rc = load().corutv_solve_corrected(h.h, ctypes.byref(p), ctypes.c_void_p(A.data_ptr()), _rowmajor_ld(A),
                                           ctypes.c_void_p(sc), ctypes.c_void_p(A_ref.data_ptr()),
                                           _rowmajor_ld(A_ref), *tail)
        _check(rc, "corutv_solve_corrected")
    info = info_wait(h) if wait else None
    return SolveResult(U, T, V, perm, info)


def solve_host(A, Phi, k: int, l: int, q: int = 0, side: str = "right", core: str = "exact", mma: str = "auto",
               want_fro2: bool = False, chunk_rows: int = 0, out=None, wait: bool = True,
               handle: Handle | None = None, orth: str = "stabilised", factor: str = "qrcp", small_f64: bool = False):
    """CoR-UTV of a HOST matrix A streamed to the GPU pass by pass (corutv_solve_host).

    A: (m, n) row-major float32 / float64 CPU tensor (page-locked, e.g.
    torch.empty(..., pin_memory=True), for full host-to-device bandwidth); it
    must stay unchanged until the solve is complete.  Phi and the outputs are
    device tensors as for solve().  chunk_rows: rows per streamed chunk (a
    multiple of 128; 0 = about 256 MiB).
    """
    import torch
    if A.is_cuda:
        raise TypeError("solve_host takes a host (CPU) A; use solve() for a device A")
    if A.dim() != 2 or A.stride(1) != 1:
        raise TypeError("A must be a row-major 2-D tensor")
    _need_cuda(Phi)
    h = handle or handle_for()
    m, n = A.shape
    code = _dt_code(A)
    fdt = torch.float64 if code == 0 else torch.float32
    if Phi.dtype != fdt:
        raise TypeError(f"Phi must be {fdt}")
    p = _params(m, n, k, l, q, side, core, code, mma, want_fro2, orth, factor, small_f64)
    if out is None:
        dev = Phi.device
        U = torch.empty((m, l), dtype=fdt, device=dev)
        T = torch.empty((l, l), dtype=torch.float64, device=dev)
        V = torch.empty((n, l), dtype=fdt, device=dev)
        perm = torch.empty((l,), dtype=torch.int32, device=dev)
    else:
        U, T, V, perm = out
    rc = load().corutv_solve_host(h.h, ctypes.byref(p), ctypes.c_void_p(A.data_ptr()), A.stride(0), int(chunk_rows),
                                  ctypes.c_void_p(Phi.data_ptr()), _rowmajor_ld(Phi), ctypes.c_void_p(U.data_ptr()),
                                  _rowmajor_ld(U), ctypes.c_void_p(T.data_ptr()), _rowmajor_ld(T),
                                  ctypes.c_void_p(V.data_ptr()), _rowmajor_ld(V), ctypes.c_void_p(perm.data_ptr()))
    _check(rc, "corutv_solve_host")
    info = info_wait(h) if wait else None
    return SolveResult(U, T, V, perm, info)


def residual_norm2(A, U, T, V, x0, k: int | None = None, iters: int = 30, handle: Handle | None = None) -> float:
    """||A - U(:,1:k) T(1:k,:) V^T||_2 by power iteration from x0 (corutv_residual_norm2).

    A (m, n), U (m, l), V (n, l), x0 (n,): device float32 / float64 of one dtype;
    T (l, l) device float64.  k defaults to l."""
    _need_cuda(A, U, T, V, x0)
    h = handle or handle_for()
    m, n = A.shape
    l = U.shape[1]
    code = _dt_code(A)
    for t in (U, V, x0):
        if t.dtype != A.dtype:
            raise TypeError("U, V and x0 must have A's dtype")
    if x0.dim() != 1 or x0.shape[0] != n or x0.stride(0) != 1:
        raise TypeError("x0 must be a contiguous vector of length n")
    out = ctypes.c_double()
    rc = load().corutv_residual_norm2(h.h, code, ctypes.c_void_p(A.data_ptr()), _rowmajor_ld(A), m, n,
                                      ctypes.c_void_p(U.data_ptr()), _rowmajor_ld(U), ctypes.c_void_p(T.data_ptr()),
                                      _rowmajor_ld(T), ctypes.c_void_p(V.data_ptr()), _rowmajor_ld(V), int(l),
                                      int(l if k is None else k), ctypes.c_void_p(x0.data_ptr()), int(iters),
                                      ctypes.byref(out))
    _check(rc, "corutv_residual_norm2")
    return out.value


class RpcaResult:
    def __init__(self, L, S, Y, info):
        self.L, self.S, self.Y, self.info = L, S, Y, info


def rpca(M, Phi, k: int, l: int, q: int, lam: float, mu0: float, rho: float, mu_bar: float, tol: float = 1e-5,
         max_iter: int = 100, side: str = "right", mma: str = "auto", out=None, handle: Handle | None = None):
    """Robust PCA by ALM-CoRUTV (Alg. 5): M (m, n) float32 on the device ~ L + S.

    Phi: (n, l) for side="right", (m, l) for side="left", float32.  out:
    optional (L, S, Y) float32 (m, n) buffers with a row pitch of a multiple
    of 4 elements.  Returns L, S, the final multiplier Y and the info
    (iterations, rank, zeta, converged)."""
    import torch
    _need_cuda(M, Phi)
    if M.dtype != torch.float32 or Phi.dtype != torch.float32:
        raise TypeError("M and Phi must be float32")
    h = handle or handle_for()
    m, n = M.shape
    if out is None:
        pitch = -(-n // 4) * 4
        L, S, Y = (torch.empty((m, pitch), dtype=torch.float32, device=M.device)[:, :n] for _ in range(3))
    else:
        L, S, Y = out
    p = RpcaParams()
    p.m, p.n, p.k, p.l, p.q = m, n, k, l, q
    p.side = SIDE[side]
    p.mma = MMA[mma]
    p.max_iter = max_iter
    p.lam, p.mu0, p.rho, p.mu_bar, p.tol = lam, mu0, rho, mu_bar, tol
    info = RpcaInfo()
    rc = load().corutv_rpca(h.h, ctypes.byref(p), ctypes.c_void_p(M.data_ptr()), _rowmajor_ld(M),
                            ctypes.c_void_p(Phi.data_ptr()), _rowmajor_ld(Phi), ctypes.c_void_p(L.data_ptr()),
                            _rowmajor_ld(L), ctypes.c_void_p(S.data_ptr()), _rowmajor_ld(S),
                            ctypes.c_void_p(Y.data_ptr()), _rowmajor_ld(Y), ctypes.byref(info))
    _check(rc, "corutv_rpca")
    if info.status != 0:
        raise CorutvError(info.status, "corutv_rpca (device)")
    return RpcaResult(L, S, Y, info)


def quantize(A, dtype: str, out=None, tile_scales=None, handle: Handle | None = None):
    """Storage conversion of a float32 device matrix (corutv_quantize):
    dtype "bf16" -> bfloat16 A (scales None); "fp8" -> (float8_e4m3fn A, float32
    tile scales of shape (ceil(m/128), ceil(n/128)), powers of two)."""
    import torch
    _need_cuda(A)
    if A.dtype != torch.float32:
        raise TypeError("quantize takes a float32 matrix")
    h = handle or handle_for()
    m, n = A.shape
    code = DTYPE[dtype]
    if code not in (2, 3):
        raise ValueError("dtype must be 'bf16' or 'fp8'")
    if out is None:
        tdt = torch.bfloat16 if code == 2 else torch.float8_e4m3fn
        ld = -(-n // 16) * 16          # 16-byte row pitch for the tensor-core passes
        out = torch.empty((m, ld), dtype=tdt, device=A.device)[:, :n]
    if code == 3 and tile_scales is None:
        tile_scales = torch.empty((-(-m // 128), -(-n // 128)), dtype=torch.float32, device=A.device)
    sc = tile_scales.data_ptr() if tile_scales is not None else 0
    rc = load().corutv_quantize(h.h, code, ctypes.c_void_p(A.data_ptr()), _rowmajor_ld(A), m, n,
                                ctypes.c_void_p(out.data_ptr()), _rowmajor_ld(out), ctypes.c_void_p(sc))
    _check(rc, "corutv_quantize")
    return (out, tile_scales) if code == 3 else (out, None)


def _fill_problem(p, it):
    """Fill a Problem struct from an item dict; returns the allocated SolveResult."""
    import torch
    A, Phi = it["A"], it["Phi"]
    _need_cuda(A, Phi, it.get("a_tile_scales"))
    m, n = A.shape
    l = int(it["l"])
    if Phi.dtype != torch.float32:
        raise TypeError("Phi must be float32")
    U = torch.empty((m, l), dtype=torch.float32, device=A.device)
    T = torch.empty((l, l), dtype=torch.float64, device=A.device)
    V = torch.empty((n, l), dtype=torch.float32, device=A.device)
    perm = torch.empty((l,), dtype=torch.int32, device=A.device)
    p.m, p.n, p.k, p.l, p.q = m, n, int(it["k"]), l, int(it.get("q", 0))
    p.side = SIDE[it.get("side", "right")]
    p.core = CORE[it.get("core", "exact")]
    p.orth = ORTH[it.get("orth", "stabilised")]
    p.a_dtype = _dt_code(A)
    p.mma = MMA[it.get("mma", "auto")]
    p.want_fro2 = 1 if it.get("want_fro2", False) else 0
    p.fuse_power = 1 if it.get("fuse_power", False) else 0
    sc = it.get("a_tile_scales")
    p.A, p.lda = A.data_ptr(), _rowmajor_ld(A)
    p.a_tile_scales = sc.data_ptr() if sc is not None else None
    p.Phi, p.ldphi = Phi.data_ptr(), _rowmajor_ld(Phi)
    p.U, p.ldu = U.data_ptr(), _rowmajor_ld(U)
    p.T, p.ldt = T.data_ptr(), _rowmajor_ld(T)
    p.V, p.ldv = V.data_ptr(), _rowmajor_ld(V)
    p.perm = perm.data_ptr()
    return SolveResult(U, T, V, perm, None)


class Server:
    """corutv_server: submit solves (item dicts as for Batch) and poll them.

    The Server keeps each request's tensors alive until it has been polled as
    finished."""

    def __init__(self, hbm_budget: int, max_slots: int = 64, queue_capacity: int = 4096, device: int | None = None):
        import torch
        self.device = torch.cuda.current_device() if device is None else device
        self.s = ctypes.c_void_p()
        _check(load().corutv_server_create(ctypes.byref(self.s), self.device, int(hbm_budget), int(max_slots),
                                           int(queue_capacity)), "corutv_server_create")
        self.live = {}

    def submit(self, item):
        """Queue one solve; returns the ticket.  Raises CorutvError (ERR_BUSY when the queue is full)."""
        p = Problem()
        res = _fill_problem(p, item)
        t = ctypes.c_uint64()
        _check(load().corutv_server_submit(self.s, ctypes.byref(p), ctypes.byref(t)), "corutv_server_submit")
        self.live[t.value] = (item, res)
        return t.value

    def poll(self, ticket: int):
        """None while pending; else (status, SolveResult) and the ticket is released."""
        info = Info()
        rc = load().corutv_server_poll(self.s, ctypes.c_uint64(ticket), ctypes.byref(info))
        if rc == PENDING:
            return None
        if rc == ERR_INVALID_ARG and ticket not in self.live:
            raise CorutvError(rc, "corutv_server_poll")
        item, res = self.live.pop(ticket)
        res.info = info
        return rc, res

    def stats(self):
        b, s, p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().corutv_server_stats(self.s, ctypes.byref(b), ctypes.byref(s), ctypes.byref(p)),
               "corutv_server_stats")
        n = ctypes.c_int64()
        _check(load().corutv_server_launches(self.s, ctypes.byref(n)), "corutv_server_launches")
        return dict(batches=b.value, solved=s.value, pending=p.value, launches=n.value)

    def close(self):
        if self.s:
            load().corutv_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A fixed set of problems for corutv_solve_batched.

    items: list of dicts with keys A (device float32 / bfloat16 / float8_e4m3fn,
    one dtype for the batch), Phi (float32, n x l for side "right", m x l for
    "left"), k, l and optionally q, side, core, orth, want_fro2, a_tile_scales, fuse_power.
    The outputs (U, T, V, perm per problem) are allocated once, so running the
    same Batch again passes an identical problem array and the library replays
    its CUDA graph of the batch."""

    def __init__(self, items, handle: Handle | None = None):
        import torch
        self.handle = handle or handle_for()
        self.items = list(items)
        self.count = len(self.items)
        self.arr = (Problem * self.count)()
        self.results = [_fill_problem(self.arr[i], it) for i, it in enumerate(self.items)]

    def workspace_size(self) -> int:
        out = ctypes.c_size_t()
        _check(load().corutv_batch_workspace_size(self.count, self.arr, ctypes.byref(out)),
               "corutv_batch_workspace_size")
        return out.value

    def run(self, wait: bool = True):
        """Enqueue the batch; with wait=True synchronise and attach each problem's info."""
        _check(load().corutv_solve_batched(self.handle.h, self.count, self.arr, None), "corutv_solve_batched")
        if wait:
            return self.wait()
        return None

    def wait(self):
        infos = (Info * self.count)()
        _check(load().corutv_batch_info_wait(self.handle.h, self.count, infos), "corutv_batch_info_wait")
        for r, inf in zip(self.results, infos):
            r.info = inf
        return self.results


def info_wait(h: Handle | None = None) -> Info:
    h = h or handle_for()
    info = Info()
    _check(load().corutv_info_wait(h.h, ctypes.byref(info)), "corutv_info_wait")
    return info


def skinny_pass(direction: str, A, Xt, l: int, mma: str = "auto", a_tile_scales=None, out=None,
                handle: Handle | None = None):
    """One streaming pass: direction "ax": Ct (l x m) = (A X)^T from Xt (l x n);
    "aty": Ct (l x n) = (A^T Y)^T from Xt (l x m).  Skinny-transposed buffers."""
    import torch
    _need_cuda(A, Xt, a_tile_scales)
    h = handle or handle_for()
    m, n = A.shape
    code = _dt_code(A)
    fdt = torch.float64 if code == 0 else torch.float32
    olen = m if direction == "ax" else n
    if out is None:
        out = torch.zeros((l, ld_for(olen)), dtype=fdt, device=A.device)
    sc = a_tile_scales.data_ptr() if a_tile_scales is not None else 0
    rc = load().corutv_pass(h.h, DIR[direction], code, MMA[mma], ctypes.c_void_p(A.data_ptr()), _rowmajor_ld(A),
                            m, n, ctypes.c_void_p(sc), ctypes.c_void_p(Xt.data_ptr()), _rowmajor_ld(Xt), int(l),
                            ctypes.c_void_p(out.data_ptr()), _rowmajor_ld(out))
    _check(rc, "corutv_pass")
    return out


def orthonormalize(Ct, length: int, l: int, want_R: bool = False, handle: Handle | None = None):
    """Shifted CholeskyQR3 of a skinny-transposed block in place; returns R if asked."""
    import torch
    _need_cuda(Ct)
    h = handle or handle_for()
    code = _dt_code(Ct)
    R = torch.empty((l, l), dtype=torch.float64, device=Ct.device) if want_R else None
    rc = load().corutv_orthonormalize(h.h, code, ctypes.c_void_p(Ct.data_ptr()), _rowmajor_ld(Ct), int(length),
                                      int(l), ctypes.c_void_p(R.data_ptr() if R is not None else 0))
    _check(rc, "corutv_orthonormalize")
    return R


def gram(Xt, Yt, length: int, l: int, handle: Handle | None = None):
    """G = X Y^T (float64, l x l) of two skinny-transposed blocks."""
    import torch
    _need_cuda(Xt, Yt)
    h = handle or handle_for()
    G = torch.empty((l, l), dtype=torch.float64, device=Xt.device)
    rc = load().corutv_gram(h.h, _dt_code(Xt), ctypes.c_void_p(Xt.data_ptr()), _rowmajor_ld(Xt),
                            ctypes.c_void_p(Yt.data_ptr()), _rowmajor_ld(Yt), int(length), int(l),
                            ctypes.c_void_p(G.data_ptr()))
    _check(rc, "corutv_gram")
    return G


def set_autotune(mode: int, cache_path: str | None = None, handle: Handle | None = None):
    """corutv_set_autotune: 1 = pick the batched plan's shapes by measurement (cached in
    cache_path, or in $CORUTV_AUTOTUNE_CACHE when cache_path is None), 0 = fixed shapes."""
    h = handle or handle_for()
    rc = load().corutv_set_autotune(h.h, int(mode), cache_path.encode() if cache_path is not None else None)
    _check(rc, "corutv_set_autotune")


def batch_tuning(handle: Handle | None = None) -> dict:
    """corutv_batch_tuning_read: the shapes of the handle's current batched plan."""
    h = handle or handle_for()
    t = BatchTuning()
    _check(load().corutv_batch_tuning_read(h.h, ctypes.byref(t)), "corutv_batch_tuning_read")
    return {"tuned": bool(t.tuned), "from_cache": bool(t.from_cache), "gram_cols": t.gram_cols,
            "split_k": t.split_k, "tc_order": t.tc_order, "tuned_ms": t.tuned_ms, "default_ms": t.default_ms}


def host_read_time(host_tensor, handle: Handle | None = None) -> float:
    """corutv_host_read_time: milliseconds for a kernel to read the page-locked host
    tensor directly (the host link as a kernel sees it)."""
    h = handle or handle_for()
    ms = ctypes.c_float()
    nbytes = host_tensor.numel() * host_tensor.element_size()
    rc = load().corutv_host_read_time(h.h, ctypes.c_void_p(host_tensor.data_ptr()), ctypes.c_size_t(nbytes),
                                      ctypes.byref(ms))
    _check(rc, "corutv_host_read_time")
    return float(ms.value)


def gram_noalloc(Xt, Yt, length: int, l: int, out, stream=None):
    """corutv_gram_noalloc: G = X Y^T into the caller's float64 (l x l) device
    tensor `out`, without any device allocation by the library (its partial
    sums use a fixed device array shared by all calls on the device)."""
    import torch
    _need_cuda(Xt, Yt, out)
    if stream is None:
        stream = torch.cuda.current_stream()
    rc = load().corutv_gram_noalloc(ctypes.c_void_p(stream.cuda_stream), _dt_code(Xt),
                                    ctypes.c_void_p(Xt.data_ptr()), _rowmajor_ld(Xt),
                                    ctypes.c_void_p(Yt.data_ptr()), _rowmajor_ld(Yt), int(length), int(l),
                                    ctypes.c_void_p(out.data_ptr()))
    _check(rc, "corutv_gram_noalloc")
    return out


def qrcp(D, k: int | None = None, dtype: str = "f64", handle: Handle | None = None):
    """QRCP of a float64 square device matrix: returns Q, R, perm, fro2 (||R||^2, ||R(:k)||^2)."""
    import torch
    _need_cuda(D)
    h = handle or handle_for()
    l = D.shape[0]
    Q = torch.empty((l, l), dtype=torch.float64, device=D.device)
    R = torch.empty((l, l), dtype=torch.float64, device=D.device)
    perm = torch.empty((l,), dtype=torch.int32, device=D.device)
    fro2 = torch.empty((2,), dtype=torch.float64, device=D.device)
    rc = load().corutv_qrcp(h.h, DTYPE[dtype], ctypes.c_void_p(D.data_ptr()), _rowmajor_ld(D), int(l),
                            int(l if k is None else k), ctypes.c_void_p(Q.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                            ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(fro2.data_ptr()))
    _check(rc, "corutv_qrcp")
    return Q, R, perm, fro2


def fro2(A, a_tile_scales=None, handle: Handle | None = None):
    """||A||_F^2 (float64 device scalar)."""
    import torch
    _need_cuda(A, a_tile_scales)
    h = handle or handle_for()
    out = torch.empty((1,), dtype=torch.float64, device=A.device)
    sc = a_tile_scales.data_ptr() if a_tile_scales is not None else 0
    m, n = A.shape
    rc = load().corutv_fro2(h.h, _dt_code(A), ctypes.c_void_p(A.data_ptr()), _rowmajor_ld(A), m, n,
                            ctypes.c_void_p(sc), ctypes.c_void_p(out.data_ptr()))
    _check(rc, "corutv_fro2")
    return out
