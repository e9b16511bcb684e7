"""Host-only checks of the C ABI: the library loads, exports every entry
point include/corutv.h declares, and rejects invalid arguments before touching
a device."""
import ctypes
import os
import re

import pytest

from paper_1810_07323_gb300 import corutv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "corutv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(corutv_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    lib = corutv.load()
    names = _declared()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), f"{name} declared in corutv.h but not exported"
    assert sorted(corutv.EXPORTS) == names


def test_version_and_status_strings():
    src = open(os.path.join(ROOT, "include", "corutv.h")).read()
    declared = int(re.search(r"#define CORUTV_ABI_VERSION (\d+)", src).group(1))
    assert corutv.version() == declared
    assert corutv.status_string(0) == "ok"
    assert "timed out" in corutv.status_string(6)
    assert corutv.status_string(999) == "unknown status"


def _ws(**kw):
    args = dict(m=100, n=80, k=5, l=10, q=0, side="right", core="exact", a_dtype="f32", mma="auto")
    args.update(kw)
    return corutv.workspace_size(**args)


@pytest.mark.parametrize("kw,status", [
    (dict(k=0), corutv.ERR_INVALID_ARG),           # 1 <= k
    (dict(k=11), corutv.ERR_INVALID_ARG),          # k <= l
    (dict(q=-1), corutv.ERR_INVALID_ARG),          # q >= 0
    (dict(l=80), corutv.ERR_SHAPE),                # l < min(m, n)
    (dict(m=1000, n=1000, l=129), corutv.ERR_SHAPE),            # l beyond the FP32 kernels
    (dict(m=1000, n=1000, l=129, a_dtype="f64"), corutv.ERR_SHAPE),  # l beyond the FP64 kernels
    (dict(a_dtype="f64", mma="tf32"), corutv.ERR_UNSUPPORTED),
    (dict(m=0), corutv.ERR_SHAPE),
    (dict(small_f64=2), corutv.ERR_INVALID_ARG),
    (dict(small_f64=1, factor="qlp"), corutv.ERR_UNSUPPORTED),   # FP64 small factorisations: QRCP only
])
def test_invalid_parameters_rejected_on_host(kw, status):
    with pytest.raises(corutv.CorutvError) as e:
        _ws(**kw)
    assert e.value.status == status


def test_null_pointers_rejected():
    lib = corutv.load()
    assert lib.corutv_create(None, None) == corutv.ERR_INVALID_ARG
    assert lib.corutv_destroy(None) == corutv.ERR_INVALID_ARG
    assert lib.corutv_info_wait(None, None) == corutv.ERR_INVALID_ARG
    assert lib.corutv_workspace_size(None, None) == corutv.ERR_INVALID_ARG
    p = corutv.Params()
    assert lib.corutv_solve(None, ctypes.byref(p), None, 0, None, None, 0, None, 0, None, 0, None, 0,
                            None) == corutv.ERR_INVALID_ARG


def test_reserved_fields_must_be_zero():
    p = corutv._params(100, 80, 5, 10, 0, "right", "exact", 1, "auto", False, "stabilised")
    p.reserved[3] = 1
    out = ctypes.c_size_t()
    assert corutv.load().corutv_workspace_size(ctypes.byref(p), ctypes.byref(out)) == corutv.ERR_INVALID_ARG


def test_device_tensors_required():
    import torch
    with pytest.raises(ValueError):
        corutv.solve(torch.zeros(10, 8), torch.zeros(8, 2), 1, 2)


def test_null_handles_rejected_by_the_newer_entry_points():
    lib = corutv.load()
    p = corutv.Params()
    out = ctypes.c_double()
    assert lib.corutv_solve_host(None, ctypes.byref(p), None, 0, 0, None, 0, None, 0, None, 0, None, 0,
                                 None) == corutv.ERR_INVALID_ARG
    assert lib.corutv_residual_norm2(None, 1, None, 0, 0, 0, None, 0, None, 0, None, 0, 1, 1, None, 1,
                                     ctypes.byref(out)) == corutv.ERR_INVALID_ARG
    assert lib.corutv_rpca(None, None, None, 0, None, 0, None, 0, None, 0, None, 0, None) == corutv.ERR_INVALID_ARG


def test_host_entry_points_check_their_tensors():
    import torch
    with pytest.raises(TypeError):
        corutv.solve_host(torch.zeros(10), torch.zeros(8, 2), 1, 2)          # A must be 2-D row-major
    with pytest.raises(TypeError):
        corutv.solve_host(torch.zeros(10, 8).t(), torch.zeros(8, 2), 1, 2)  # not row-major
    with pytest.raises(ValueError):
        corutv.residual_norm2(torch.zeros(10, 8), torch.zeros(10, 2), torch.zeros(2, 2, dtype=torch.float64),
                              torch.zeros(8, 2), torch.zeros(8))             # device tensors required


def _problem(m=700, n=300, k=6, l=14, q=1, dtype="f32", lda=None, fuse=0, orth="stabilised", scales=True,
             a_addr=0x10000):
    """A batched problem descriptor with placeholder (never dereferenced) device addresses."""
    p = corutv.Problem()
    p.m, p.n, p.k, p.l, p.q = m, n, k, l, q
    p.side, p.core, p.orth = corutv.SIDE["right"], corutv.CORE["exact"], corutv.ORTH[orth]
    p.a_dtype = corutv.DTYPE[dtype]
    p.mma, p.want_fro2, p.fuse_power = 0, 1, fuse
    p.A = a_addr
    p.lda = n if lda is None else lda
    p.a_tile_scales = 0x20000 if (dtype == "fp8" and scales) else None
    p.Phi, p.ldphi = 0x30000, l
    p.U, p.ldu, p.T, p.ldt, p.V, p.ldv, p.perm = 0x40000, l, 0x50000, l, 0x60000, l, 0x70000
    return p


def _batch_ws(probs):
    arr = (corutv.Problem * len(probs))(*probs)
    out = ctypes.c_size_t()
    rc = corutv.load().corutv_batch_workspace_size(len(probs), arr, ctypes.byref(out))
    return rc, out.value


def test_batch_workspace_size_on_the_host():
    """The batched plan is made on the host (no device needed): its size is deterministic,
    grows with the problems it holds, and counts every problem of a mixed set."""
    rc1, one = _batch_ws([_problem()])
    rc1b, one_b = _batch_ws([_problem()])
    rc2, two = _batch_ws([_problem(), _problem(m=4096, n=2048, k=30, l=40)])
    rc3, bf = _batch_ws([_problem(dtype="bf16", n=304), _problem(dtype="fp8", n=304)])
    assert rc1 == rc1b == rc2 == rc3 == corutv.OK
    assert one == one_b > 0 and two > one and bf > 0


@pytest.mark.parametrize("kw,status", [
    (dict(k=15, l=14), corutv.ERR_INVALID_ARG),              # k > l
    (dict(l=300), corutv.ERR_SHAPE),                         # l >= min(m, n)
    (dict(q=-1), corutv.ERR_INVALID_ARG),
    (dict(lda=200), corutv.ERR_SHAPE),                       # lda < n
    (dict(dtype="fp8", scales=False), corutv.ERR_INVALID_ARG),
    (dict(fuse=2), corutv.ERR_INVALID_ARG),
    (dict(orth="literal"), corutv.ERR_UNSUPPORTED),          # Alg. 3 as printed: single solves only
])
def test_batch_problem_validation_on_the_host(kw, status):
    rc, _ = _batch_ws([_problem(), _problem(**kw)])
    assert rc == status
