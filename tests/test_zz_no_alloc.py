"""corutv_gram_noalloc: the Gram product for callers that must not allocate
device memory after start-up (its partial sums live in a fixed device array).
Checked through the C ABI on two calls in a row, which share that array,
against the FP64 product of the same inputs formed directly and against
corutv_gram (the allocating entry point); the first case splits its columns
over fewer partial blocks than corutv_gram does (the array holds 32)."""
import numpy as np
import pytest

from synth import counter as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1810_07323_gb300 import corutv


def _st(seed, l, length, dtype):
    host = C.normal_block_np(seed, length, 0, l, 0, length)
    buf = torch.zeros((l, corutv.ld_for(length)), dtype=dtype, device="cuda")
    buf[:, :length] = torch.tensor(host, dtype=dtype, device="cuda")
    return buf


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_gram_noalloc_matches_gram_twice(dt):
    l_len = [(120, 20000), (37, 3001)]          # two different calls in a row
    outs = []
    for i, (l, length) in enumerate(l_len):
        Xt = _st(100 + i, l, length, dt)
        Yt = _st(200 + i, l, length, dt)
        G = torch.empty((l, l), dtype=torch.float64, device="cuda")
        corutv.gram_noalloc(Xt, Yt, length, l, G)
        outs.append((Xt, Yt, l, length, G))
    torch.cuda.synchronize()
    # FP32 partial sums over different column ranges: agreement to a few FP32 ulps
    # of sum |x||y| (FP64: to a few FP64 ulps)
    tol = 1e-6 if dt == torch.float32 else 1e-14
    for Xt, Yt, l, length, G in outs:
        x, y = Xt[:, :length].double(), Yt[:, :length].double()
        scale = x.abs() @ y.abs().T
        direct = x @ y.T                               # the FP64 product of the same inputs
        assert torch.all((G - direct).abs() <= tol * scale + 1e-300), float(((G - direct).abs() / scale).max())
        ref = corutv.gram(Xt, Yt, length, l)           # the allocating entry point
        assert torch.all((G - ref).abs() <= tol * scale + 1e-300), float(((G - ref).abs() / scale).max())


def test_gram_noalloc_allocates_nothing():
    """After a first call (which may load the module on the device), further calls
    leave torch's allocator untouched and give the same result."""
    l, length = 64, 5000
    Xt = _st(300, l, length, torch.float32)
    G1 = torch.empty((l, l), dtype=torch.float64, device="cuda")
    G2 = torch.empty_like(G1)
    corutv.gram_noalloc(Xt, Xt, length, l, G1)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    corutv.gram_noalloc(Xt, Xt, length, l, G2)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    assert torch.equal(G1, G2)


def test_gram_noalloc_rejects_oversize():
    Xt = torch.zeros((129, 64), device="cuda")
    G = torch.empty((129, 129), dtype=torch.float64, device="cuda")
    with pytest.raises(corutv.CorutvError) as e:
        corutv.gram_noalloc(Xt, Xt, 64, 129, G)
    assert e.value.status == corutv.ERR_SHAPE
