"""GPU tests of the serving queue (corutv_server_*): every BF16 request's result
equals the same problem solved alone (bit for bit: the grouped kind::f16
passes cut each problem into work units of its own -- output tile and K range
-- and add split tiles in range order, and the other batched kernels compute
each problem independently of the others in its batch; FP32 batches on the
TF32 tensor-core pass split their passes by batch, so there results agree to
rounding), the queue reports
ERR_BUSY when full and never blocks, oversized requests fail with ERR_OOM,
invalid ones are refused at submission, and results agree with the FP64
oracle on sampled requests."""
import time

import numpy as np
import pytest

from oracle import corutv_oracle as O
from synth import counter as C
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1810_07323_gb300 import corutv

SIZES = [(1024, 512), (2048, 512), (3000, 200)]


def _item(i, kind="bf16"):
    m, n = SIZES[i % 3]
    k = (5, 20, 50)[(i // 3) % 3]
    l = k + 10
    q = i % 2
    content = W.LowRankSparse(m, n, 5, 0.05, 10.0, C.stream_seed(500, i))
    A = content.dense_t(device="cuda", dtype=torch.float32)
    if kind == "bf16":
        A = A.to(torch.bfloat16)
    phi = C.normal_block_t(C.stream_seed(501, i), l, 0, n, 0, l, device="cuda").float()
    return dict(A=A, Phi=phi, k=k, l=l, q=q, want_fro2=True)


def _drain(srv, tickets, timeout=60.0):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets):
        for t in tickets:
            if t in done:
                continue
            r = srv.poll(t)
            if r is not None:
                done[t] = r
        assert time.time() - t0 < timeout, "requests did not finish"
        time.sleep(1e-4)
    return done


def test_server_results_equal_solved_alone():
    items = [_item(i) for i in range(24)]
    srv = corutv.Server(hbm_budget=4 << 30, max_slots=8)
    tickets = [srv.submit(it) for it in items]
    done = _drain(srv, tickets)
    st = srv.stats()
    srv.close()
    assert st["solved"] == len(items) and st["batches"] >= 3     # several batches, up to 8 requests each
    assert st["launches"] >= 10 * st["batches"]                  # library kernels ran for every batch
    for t, it in zip(tickets, items):
        rc, res = done[t]
        assert rc == corutv.OK and res.info.status == 0
        alone = corutv.Batch([it]).run()[0]
        assert torch.equal(res.U, alone.U) and torch.equal(res.T, alone.T)
        assert torch.equal(res.V, alone.V) and torch.equal(res.perm, alone.perm)
        assert res.info.fro2_T == alone.info.fro2_T


def test_server_parity_with_oracle_sampled():
    items = [_item(i, kind="f32") for i in range(6)]
    srv = corutv.Server(hbm_budget=4 << 30, max_slots=4)
    tickets = [srv.submit(it) for it in items]
    done = _drain(srv, tickets)
    srv.close()
    for t, it in zip(tickets, items):
        rc, res = done[t]
        assert rc == corutv.OK
        A = it["A"].double().cpu().numpy()
        ref = O.corutv(A, it["Phi"].double().cpu().numpy(), it["k"], it["l"], it["q"])
        rho = O.factor_distance(res.U.double().cpu().numpy(), res.T.cpu().numpy(), res.V.double().cpu().numpy(),
                                ref["U"], ref["T"], ref["V"])
        assert rho < 1e-3, rho       # FP32 rows TMA can read: grouped TF32 tensor-core passes


def test_server_queue_full_is_busy_and_never_blocks():
    # large requests keep both batch slots busy while the 2-entry queue fills
    big = []
    for i in range(12):
        m, n = 8192, 2048
        A = torch.randn((m, n), device="cuda").to(torch.bfloat16)
        phi = torch.randn((n, 60), device="cuda")
        big.append(dict(A=A, Phi=phi, k=50, l=60, q=1))
    srv = corutv.Server(hbm_budget=8 << 30, max_slots=1, queue_capacity=2)
    tickets, busy = [], 0
    t0 = time.perf_counter()
    for it in big:
        try:
            tickets.append(srv.submit(it))
        except corutv.CorutvError as e:
            assert e.status == corutv.ERR_BUSY
            busy += 1
    assert time.perf_counter() - t0 < 1.0          # submissions did not wait for the GPU
    assert busy > 0
    done = _drain(srv, tickets)
    srv.close()
    assert all(rc == corutv.OK for rc, _ in done.values())


def test_server_oversized_request_fails_with_oom():
    it = _item(0)
    srv = corutv.Server(hbm_budget=1 << 20, max_slots=4)     # 1 MiB: smaller than A alone
    t = srv.submit(it)
    rc, _ = _drain(srv, [t])[t]
    srv.close()
    assert rc == corutv.ERR_OOM


def test_server_invalid_request_refused_at_submit():
    it = _item(0)
    it["k"] = it["l"] + 1
    srv = corutv.Server(hbm_budget=1 << 30)
    with pytest.raises(corutv.CorutvError) as e:
        srv.submit(it)
    srv.close()
    assert e.value.status == corutv.ERR_INVALID_ARG
