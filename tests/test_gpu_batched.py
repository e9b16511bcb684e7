"""GPU parity of corutv_solve_batched (grouped launches over many problems of
different shapes) with the FP64 oracle run on each problem's stored values,
replay determinism of the captured batch, and the 1024-problem workload
(m ~ U{256..4096}, n ~ U{128..2048}, l = r + 8, q = 1) on sampled problems.

Batches of FP32 A whose rows TMA can address run the passes as grouped TF32
tensor-core launches (bound rho <= 1e-3, as corutv_solve with mma = tf32).
BF16 / FP8 problems whose rows TMA can address run theirs as grouped kind::f16
launches (BF16 A exact, the sketch split into two BF16 parts, FP32
accumulation) whose work units depend on the problem alone, so each result is
the same bits alone and in any batch; the rest accumulate FP32 products on the
CUDA cores.  Both forms hold rho <= 1e-4, the factorisations running in FP32
as in corutv_solve with mma = SIMT."""
import numpy as np
import pytest

from oracle import corutv_oracle as O
from oracle import precision as P
from synth import counter as C
from synth import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1810_07323_gb300 import corutv

TOL = 1e-4


def _lowrank_sparse(seed, m, n, r):
    return W.LowRankSparse(m, n, r, 0.05, 10.0, seed).dense()


def _item(A32, phi, k, l, q=1, side="right", core="exact", orth="stabilised", want_fro2=True, kind="f32"):
    m, n = A32.shape
    if kind == "f32":
        Ad = torch.tensor(A32, dtype=torch.float32, device="cuda")
        S, Aq = None, A32.astype(np.float64)
    elif kind == "bf16":
        v = P.bf16_round(A32)
        Ad = torch.tensor(v).to(torch.bfloat16).cuda()
        S, Aq = None, v.astype(np.float64)
    else:
        vals, sc = P.quantize_fp8(A32)
        Ad = torch.tensor(vals.astype(np.float32)).to(torch.float8_e4m3fn).cuda()
        S, Aq = torch.tensor(sc, dtype=torch.float32, device="cuda"), P.dequantize_fp8(vals, sc)
    it = dict(A=Ad, Phi=torch.tensor(phi, dtype=torch.float32, device="cuda"), k=k, l=l, q=q, side=side,
              core=core, orth=orth, want_fro2=want_fro2)
    if S is not None:
        it["a_tile_scales"] = S
    return it, Aq


MIXED = [
    # m, n, r, k, l, q, side, core, orth
    (700, 300, 6, 6, 14, 1, "right", "exact", "stabilised"),
    (256, 1100, 10, 10, 18, 1, "left", "exact", "stabilised"),
    (1500, 900, 20, 20, 28, 2, "right", "sketch", "stabilised"),
    (333, 129, 4, 4, 12, 0, "right", "exact", "stabilised"),
    (2048, 2047, 32, 32, 40, 1, "right", "exact", "strict"),
    (640, 1900, 12, 12, 20, 2, "left", "sketch", "stabilised"),
    (4096, 128, 30, 30, 38, 1, "right", "exact", "stabilised"),
    (1000, 1000, 60, 60, 100, 0, "right", "exact", "stabilised"),     # l = 100: the 128-row kernels
]


def _check(res, Aq, phi, k, l, q, side, core):
    U = res.U.double().cpu().numpy()
    T = res.T.cpu().numpy()
    V = res.V.double().cpu().numpy()
    perm = res.perm.cpu().numpy()
    ref = O.corutv(Aq, phi.astype(np.float64), k, l, q, side=side)
    rho = O.factor_distance(U, T, V, ref["U"], ref["T"], ref["V"])
    tri = np.tril(T, -1) if side == "right" else np.triu(T, 1)
    assert np.abs(tri).max() == 0.0
    assert np.all(np.diag(T) >= 0) and sorted(perm) == list(range(l))
    assert O.orthonormality_error(U) < 5e-5 and O.orthonormality_error(V) < 5e-5
    return rho


@pytest.mark.parametrize("kind", ["f32", "bf16", "fp8"])
def test_batched_mixed_parity(kind):
    items, refs = [], []
    for i, (m, n, r, k, l, q, side, core, orth) in enumerate(MIXED):
        A = _lowrank_sparse(C.stream_seed(77, i), m, n, r).astype(np.float32)
        phi = C.normal_block_np(C.stream_seed(78, i), l, 0, m if side == "left" else n, 0, l)
        it, Aq = _item(A, phi, k, l, q, side, core, orth, kind=kind)
        items.append(it)
        refs.append((Aq, phi, k, l, q, side, core))
    b = corutv.Batch(items)
    res = b.run()
    for i, (r, (Aq, phi, k, l, q, side, core)) in enumerate(zip(res, refs)):
        assert r.info.status == 0
        rho = _check(r, Aq, phi, k, l, q, side, core)
        print(f"{kind} problem {i} {MIXED[i][:2]}: rho={rho:.3e}")
        assert rho < TOL, (i, rho)
        a2 = float(np.sum(Aq ** 2))
        assert abs(r.info.fro2_A - a2) < 1e-6 * a2
        assert abs(r.info.fro2_T - float(np.sum(r.T.cpu().numpy() ** 2))) < 1e-9 * a2
        assert r.info.passes_over_A == 2 * (q + 1) + (1 if core == "exact" else 0)


SPLIT = [
    # SIMT passes whose reduction length K exceeds 2 x 2048 run as K ranges summed by the last CTA of
    # each tile: C2 = A^T Q1 over 9000 rows, C2 = A Q1 over 8500 columns (LEFT), C1 and the core
    # over 9000 columns (with ||A||^2 folded over the split blocks), 20 ranges over 40000 rows
    (9000, 150, 8, 8, 16, 1, "right", "exact", "stabilised"),
    (200, 8500, 6, 6, 14, 1, "left", "exact", "stabilised"),
    (300, 9000, 10, 10, 18, 0, "right", "exact", "stabilised"),
    (40000, 130, 5, 5, 12, 1, "right", "sketch", "stabilised"),
    (700, 300, 6, 6, 14, 1, "right", "exact", "stabilised"),
]


@pytest.mark.parametrize("kind", ["f32simt", "bf16", "fp8"])
def test_batched_split_k_parity(kind):
    items, refs = [], []
    for i, (m, n, r, k, l, q, side, core, orth) in enumerate(SPLIT):
        A = _lowrank_sparse(C.stream_seed(81, i), m, n, r).astype(np.float32)
        phi = C.normal_block_np(C.stream_seed(82, i), l, 0, m if side == "left" else n, 0, l)
        it, Aq = _item(A, phi, k, l, q, side, core, orth, kind="f32" if kind == "f32simt" else kind)
        if kind == "f32simt":
            it["mma"] = "simt"
        items.append(it)
        refs.append((Aq, phi, k, l, q, side, core))
    b = corutv.Batch(items)
    outs = []
    for run in range(3):          # direct launches, capture, replay: identical (the range sums are ordered)
        res = b.run()
        outs.append([(x.U.clone(), x.T.clone(), x.V.clone()) for x in res])
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert all(torch.equal(x, y) for x, y in zip(a, c))
    for i, (r, (Aq, phi, k, l, q, side, core)) in enumerate(zip(res, refs)):
        assert r.info.status == 0
        rho = _check(r, Aq, phi, k, l, q, side, core)
        print(f"{kind} split problem {i} {SPLIT[i][:2]}: rho={rho:.3e}")
        assert rho < TOL, (i, rho)
        a2 = float(np.sum(Aq ** 2))
        assert abs(r.info.fro2_A - a2) < 1e-6 * a2


F16 = [
    # BF16 / FP8 rows TMA can address (n a multiple of 16): grouped kind::f16 passes.  K cut into
    # ranges of 2048 k (C2 over 9216 and 40000 rows, the LEFT problem's C2 over 8704 columns, C1
    # and the core over 9216 columns with ||A||^2 folded per unit), ragged tiles, l = 128, both
    # sides and cores; the last problem's rows (129 elements) take the CUDA-core pass in the same batch
    (9216, 160, 8, 8, 16, 1, "right", "exact", "stabilised"),
    (208, 8704, 6, 6, 14, 1, "left", "exact", "stabilised"),
    (304, 9216, 10, 10, 18, 0, "right", "exact", "stabilised"),
    (40000, 144, 5, 5, 12, 1, "right", "sketch", "stabilised"),
    (1000, 1008, 60, 60, 128, 2, "right", "exact", "strict"),
    (700, 304, 6, 6, 14, 1, "right", "exact", "stabilised"),
    (333, 129, 4, 4, 12, 0, "right", "exact", "stabilised"),
]


@pytest.mark.parametrize("kind", ["bf16", "fp8"])
def test_batched_f16_grouped_parity_and_alone(kind):
    """Grouped kind::f16 passes: parity with the oracle on the stored values, ||A||^2 from
    the first pass's units, replays bit-identical, and every problem's factors the same bits
    when solved alone as in the batch."""
    items, refs = [], []
    for i, (m, n, r, k, l, q, side, core, orth) in enumerate(F16):
        A = _lowrank_sparse(C.stream_seed(83, i), m, n, r).astype(np.float32)
        phi = C.normal_block_np(C.stream_seed(84, i), l, 0, m if side == "left" else n, 0, l)
        it, Aq = _item(A, phi, k, l, q, side, core, orth, kind=kind)
        items.append(it)
        refs.append((Aq, phi, k, l, q, side, core))
    b = corutv.Batch(items)
    outs = []
    for _ in range(3):            # direct launches, capture, replay
        res = b.run()
        outs.append([(x.U.clone(), x.T.clone(), x.V.clone(), x.perm.clone()) for x in res])
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert all(torch.equal(x, y) for x, y in zip(a, c))
    for i, (r, (Aq, phi, k, l, q, side, core)) in enumerate(zip(res, refs)):
        assert r.info.status == 0
        rho = _check(r, Aq, phi, k, l, q, side, core)
        print(f"{kind} f16 problem {i} {F16[i][:2]}: rho={rho:.3e}")
        assert rho < TOL, (i, rho)
        a2 = float(np.sum(Aq ** 2))
        assert abs(r.info.fro2_A - a2) < 1e-6 * a2
        assert r.info.passes_over_A == 2 * (q + 1) + (1 if core == "exact" else 0)
    for i, (it, r) in enumerate(zip(items, res)):
        alone = corutv.Batch([it]).run()[0]
        assert torch.equal(alone.U, r.U) and torch.equal(alone.T, r.T), i
        assert torch.equal(alone.V, r.V) and torch.equal(alone.perm, r.perm), i
        assert alone.info.fro2_A == r.info.fro2_A and alone.info.fro2_T == r.info.fro2_T, i


def test_batched_replay_is_identical():
    """First run (direct launches), second (captured into a CUDA graph) and third
    (graph replay) give bit-identical factors."""
    items = []
    for i, (m, n, r, k, l, q, side, core, orth) in enumerate(MIXED[:6]):
        A = _lowrank_sparse(C.stream_seed(90, i), m, n, r).astype(np.float32)
        phi = C.normal_block_np(C.stream_seed(91, i), l, 0, m if side == "left" else n, 0, l)
        items.append(_item(A, phi, k, l, q, side, core, orth)[0])
    b = corutv.Batch(items)
    outs = []
    for _ in range(3):
        res = b.run()
        outs.append([(r.U.clone(), r.T.clone(), r.V.clone(), r.perm.clone()) for r in res])
        assert all(r.info.status == 0 for r in res)
    for run in outs[1:]:
        for a, c in zip(outs[0], run):
            assert all(torch.equal(x, y) for x, y in zip(a, c))


def test_batched_single_problem_matches_solve():
    """A batch of one agrees with corutv_solve (SIMT passes) to FP32 rounding."""
    A = _lowrank_sparse(5, 1200, 700, 15).astype(np.float32)
    phi = C.normal_block_np(6, 23, 0, 700, 0, 23)
    it, _ = _item(A, phi, 15, 23, 1)
    it["mma"] = "simt"
    r = corutv.Batch([it]).run()[0]
    s = corutv.solve(it["A"], it["Phi"], 15, 23, 1, mma="simt")
    rho = O.factor_distance(r.U.double().cpu().numpy(), r.T.cpu().numpy(), r.V.double().cpu().numpy(),
                            s.U.double().cpu().numpy(), s.T.cpu().numpy(), s.V.double().cpu().numpy())
    assert rho < 1e-5, rho


def _padded(A32):
    """Device FP32 copy with a 16-byte row pitch (the tensor-core passes read rows by TMA)."""
    m, n = A32.shape
    buf = torch.zeros((m, -(-n // 4) * 4 + 4), dtype=torch.float32, device="cuda")[:, :n]
    buf.copy_(torch.tensor(A32, device="cuda"))
    return buf


@pytest.mark.parametrize("q_all", [None, 0])
def test_batched_tensor_core_parity(q_all):
    """FP32 batches whose rows TMA can address run every pass as one grouped
    TF32 tensor-core launch (operands rounded to nearest): rho <= 1e-3 as for
    corutv_solve with mma = tf32; ||A||^2 fused into the first pass."""
    items, refs = [], []
    for i, (m, n, r, k, l, q, side, core, orth) in enumerate(MIXED):
        q = q if q_all is None else q_all
        A = _lowrank_sparse(C.stream_seed(80, i), m, n, r).astype(np.float32)
        phi = C.normal_block_np(C.stream_seed(81, i), l, 0, m if side == "left" else n, 0, l)
        items.append(dict(A=_padded(A), Phi=torch.tensor(phi, dtype=torch.float32, device="cuda"), k=k, l=l, q=q,
                          side=side, core=core, orth=orth, want_fro2=True, mma="tf32"))
        refs.append((A.astype(np.float64), phi, k, l, q, side, core))
    b = corutv.Batch(items)
    res = b.run()
    for i, (r, (Aq, phi, k, l, q, side, core)) in enumerate(zip(res, refs)):
        assert r.info.status == 0
        rho = _check(r, Aq, phi, k, l, q, side, core)
        print(f"tc problem {i} {MIXED[i][:2]}: rho={rho:.3e}")
        assert rho < 1e-3, (i, rho)
        a2 = float(np.sum(Aq ** 2))
        assert abs(r.info.fro2_A - a2) < 1e-6 * a2
        assert r.info.passes_over_A == 2 * (q + 1) + (1 if core == "exact" else 0)
    # deterministic: the same batch again (captured, then replayed) gives the same bits
    U0 = [r.U.clone() for r in res]
    for _ in range(2):
        again = b.run()
        assert all(torch.equal(a, r.U) for a, r in zip(U0, again))


def test_batched_tf32_needs_aligned_rows():
    A = torch.zeros((100, 81), device="cuda")                  # 324-byte rows
    phi = torch.zeros((81, 10), device="cuda")
    with pytest.raises(corutv.CorutvError) as e:
        corutv.Batch([dict(A=A, Phi=phi, k=5, l=10, mma="tf32")]).run()
    assert e.value.status == corutv.ERR_ALIGN


def test_batched_invalid_arguments():
    A = torch.zeros((100, 80), device="cuda")
    phi = torch.zeros((80, 10), device="cuda")
    with pytest.raises(corutv.CorutvError) as e:
        corutv.Batch([dict(A=A, Phi=phi, k=11, l=10)]).run()
    assert e.value.status == corutv.ERR_INVALID_ARG
    with pytest.raises(corutv.CorutvError) as e:
        corutv.Batch([dict(A=A, Phi=torch.zeros((80, 80), device="cuda"), k=5, l=80)]).run()
    assert e.value.status == corutv.ERR_SHAPE
    A64 = torch.zeros((100, 80), dtype=torch.float64, device="cuda")
    with pytest.raises(corutv.CorutvError) as e:
        corutv.Batch([dict(A=A64, Phi=phi, k=5, l=10)]).run()
    assert e.value.status == corutv.ERR_UNSUPPORTED
    Ab = torch.zeros((100, 80), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(corutv.CorutvError) as e:           # one storage dtype per batch
        corutv.Batch([dict(A=A, Phi=phi, k=5, l=10), dict(A=Ab, Phi=phi, k=5, l=10)]).run()
    assert e.value.status == corutv.ERR_UNSUPPORTED


def _config4_items(probs):
    items = []
    for p in probs:
        side = "left" if p.m < p.n else "right"
        dense = p.content.dense_t(device="cuda", dtype=torch.float32)
        A = torch.zeros((p.m, -(-p.n // 4) * 4), dtype=torch.float32, device="cuda")[:, :p.n]
        A.copy_(dense)
        phi = W.problem_phi_t(p, p.m if side == "left" else p.n, device="cuda").float()
        items.append(dict(A=A, Phi=phi, k=p.k, l=p.l, q=p.q, side=side, want_fro2=True))
    return items


@pytest.mark.slow
def test_config4_full_batch_sampled():
    """The 1024-problem workload in one batched call: every problem's structure
    and Pythagorean readout, 24 sampled problems against the oracle."""
    probs = W.batch_config4()
    items = _config4_items(probs)
    b = corutv.Batch(items)
    res = b.run()
    rng = np.random.default_rng(0)
    sample = set(rng.choice(len(probs), 24, replace=False).tolist())
    for i, (p, it, r) in enumerate(zip(probs, items, res)):
        assert r.info.status == 0
        T = r.T
        side = it["side"]
        tri = torch.tril(T, -1) if side == "right" else torch.triu(T, 1)
        assert float(tri.abs().max()) == 0.0
        U, V = r.U.double(), r.V.double()
        eye = torch.eye(p.l, dtype=torch.float64, device="cuda")
        assert float((U.T @ U - eye).abs().max()) < 5e-5
        assert float((V.T @ V - eye).abs().max()) < 5e-5
        A = it["A"].double()
        res2 = float(((A - (U @ T) @ V.T) ** 2).sum())
        a2 = r.info.fro2_A
        assert abs(a2 - float((A ** 2).sum())) < 1e-6 * a2
        # exact core: ||A - U T V^T||^2 = ||A||^2 - ||T||^2, up to the TF32 error of the core
        # (|dT| <= 2^-10 |T| per the pass bound, so within 2 * 2^-10 ||A||^2)
        assert abs((a2 - r.info.fro2_T) - res2) < 2e-3 * a2
        if i in sample:
            Aq = it["A"].double().cpu().numpy()
            phi = it["Phi"].double().cpu().numpy()
            ref = O.corutv(Aq, phi, p.k, p.l, p.q, side=side)
            rho = O.factor_distance(U.cpu().numpy(), T.cpu().numpy(), V.cpu().numpy(), ref["U"], ref["T"],
                                    ref["V"])
            assert rho < 1e-3, (i, rho)          # TF32 tensor-core passes


@pytest.mark.parametrize("kind", ["f32", "bf16"])
def test_autotune_plans_agree_and_cache_round_trip(kind, tmp_path):
    """The autotuner searches the plan's shapes on the first call, writes its choice to the
    JSON cache, and a second handle reads it back without searching.  Tuned and fixed plans
    give the same factorisations up to the order of FP32 sums (rho <= 1e-5 between them, and
    each within the oracle bound); the same plan replayed is bit-identical."""
    import json
    items, refs = [], []
    for i, (m, n, r, k, l, q, side, core, orth) in enumerate(MIXED + SPLIT):
        A = _lowrank_sparse(C.stream_seed(91, i), m, n, r).astype(np.float32)
        phi = C.normal_block_np(C.stream_seed(92, i), l, 0, m if side == "left" else n, 0, l)
        it, Aq = _item(A, phi, k, l, q, side, core, orth, kind=kind)
        items.append(it)
        refs.append((Aq, phi, k, l, q, side, core))
    cache = str(tmp_path / "tune.json")

    def factors(res):
        return [(x.U.double().cpu().numpy(), x.T.cpu().numpy(), x.V.double().cpu().numpy()) for x in res]

    h0 = corutv.Handle()
    fixed = factors(corutv.Batch(items, handle=h0).run())
    assert not corutv.batch_tuning(h0)["tuned"]

    h1 = corutv.Handle()
    corutv.set_autotune(1, cache, handle=h1)
    b1 = corutv.Batch(items, handle=h1)
    tuned = factors(b1.run())
    t1 = corutv.batch_tuning(h1)
    print(kind, t1)
    assert t1["tuned"] and not t1["from_cache"] and 0 < t1["tuned_ms"] <= t1["default_ms"]
    entries = json.load(open(cache))["entries"]
    assert len(entries) == 1 and entries[0]["gram_cols"] == t1["gram_cols"]
    again = factors(b1.run())                          # graph replay of the tuned plan
    for a, b in zip(tuned, again):
        assert all(np.array_equal(x, y) for x, y in zip(a, b))

    h2 = corutv.Handle()
    corutv.set_autotune(1, cache, handle=h2)
    cached = factors(corutv.Batch(items, handle=h2).run())
    t2 = corutv.batch_tuning(h2)
    assert t2["tuned"] and t2["from_cache"]
    assert (t2["gram_cols"], t2["split_k"], t2["tc_order"]) == (t1["gram_cols"], t1["split_k"], t1["tc_order"])
    for a, b in zip(tuned, cached):                    # same shapes: the same arithmetic
        assert all(np.array_equal(x, y) for x, y in zip(a, b))

    for i, ((U0, T0, V0), (U1, T1, V1), (Aq, phi, k, l, q, side, core)) in enumerate(zip(fixed, tuned, refs)):
        assert O.factor_distance(U1, T1, V1, U0, T0, V0) < 1e-5, i
        ref = O.corutv(Aq, phi.astype(np.float64), k, l, q, side=side)
        assert O.factor_distance(U1, T1, V1, ref["U"], ref["T"], ref["V"]) < TOL, i


def _fused_items(kind, seed):
    """The F16 set (BF16 rows TMA can address) or the MIXED set in FP32 with 16-byte row pitch
    (grouped TF32 passes), each problem asking for fused power steps."""
    rows = F16 if kind == "bf16" else MIXED
    items, refs = [], []
    for i, (m, n, r, k, l, q, side, core, orth) in enumerate(rows):
        A = _lowrank_sparse(C.stream_seed(seed, i), m, n, r).astype(np.float32)
        phi = C.normal_block_np(C.stream_seed(seed + 1, i), l, 0, m if side == "left" else n, 0, l)
        if kind == "bf16":
            it, Aq = _item(A, phi, k, l, q, side, core, orth, kind="bf16")
        else:
            it = dict(A=_padded(A), Phi=torch.tensor(phi, dtype=torch.float32, device="cuda"), k=k, l=l, q=q,
                      side=side, core=core, orth=orth, want_fro2=True)
            Aq = A.astype(np.float64)
        it["fuse_power"] = True
        items.append(it)
        refs.append((Aq, phi, k, l, q, side, core))
    return rows, items, refs


@pytest.mark.parametrize("kind", ["bf16", "f32"])
def test_batched_fused_power_steps(kind):
    """Fused power steps (Alg. 3 steps 3-4 with A read once per step): W = op2(A) C1 right after
    C1 while A is in L2, C2 = W R1^-1.  Parity with the oracle within the batched bounds,
    A streamed from HBM q + 1 (+ 1) times on the tensor-core engines, replays bit-identical,
    and (BF16) every problem the same bits alone as in the batch."""
    rows, items, refs = _fused_items(kind, 95)
    b = corutv.Batch(items)
    outs = []
    for _ in range(3):
        res = b.run()
        outs.append([(x.U.clone(), x.T.clone(), x.V.clone()) for x in res])
    for o in outs[1:]:
        for a, c in zip(outs[0], o):
            assert all(torch.equal(x, y) for x, y in zip(a, c))
    tol = TOL if kind == "bf16" else 1e-3
    for i, (r, it, (Aq, phi, k, l, q, side, core)) in enumerate(zip(res, items, refs)):
        assert r.info.status == 0
        rho = _check(r, Aq, phi, k, l, q, side, core)
        m, n = Aq.shape
        tc = kind == "f32" or (n % 8 == 0)                  # rows TMA can address: a tensor-core engine
        passes = 2 * (q + 1) + (1 if core == "exact" else 0)
        assert r.info.passes_over_A == passes
        assert r.info.hbm_passes_over_A == (passes - (q + 1) if tc else passes), (i, r.info.hbm_passes_over_A)
        print(f"{kind} fused problem {i} {rows[i][:2]} q={q}: rho={rho:.3e}")
        assert rho < tol, (i, rho)
        a2 = float(np.sum(Aq ** 2))
        assert abs(r.info.fro2_A - a2) < 1e-6 * a2
    if kind == "bf16":
        for i, (it, r) in enumerate(zip(items, res)):
            alone = corutv.Batch([it]).run()[0]
            assert torch.equal(alone.U, r.U) and torch.equal(alone.T, r.T), i
            assert torch.equal(alone.V, r.V), i


def test_batched_fuse_power_flag_is_checked():
    A = torch.zeros((100, 80), device="cuda")
    phi = torch.zeros((80, 10), device="cuda")
    b = corutv.Batch([dict(A=A, Phi=phi, k=5, l=10)])
    b.arr[0].fuse_power = 2
    with pytest.raises(corutv.CorutvError) as e:
        b.run()
    assert e.value.status == corutv.ERR_INVALID_ARG


@pytest.mark.parametrize("kind", ["f32", "bf16"])
def test_batched_trace_times_the_pass_kernels_alone(kind):
    """A traced batch of TMA-addressable problems records, for every grouped pass, an event
    pair around the pass kernel besides the one around its phase (operand preparation and
    split-tile reduction included)."""
    shapes = [(700, 304, 6, 6, 14, 1, "right", "exact", "stabilised"),     # rows of 16-byte multiples
              (512, 1104, 10, 10, 18, 1, "left", "exact", "stabilised"),
              (1500, 896, 20, 20, 28, 2, "right", "sketch", "stabilised")]
    items = []
    for i, (m, n, r, k, l, q, side, core, orth) in enumerate(shapes):
        A = _lowrank_sparse(C.stream_seed(95, i), m, n, r).astype(np.float32)
        phi = C.normal_block_np(C.stream_seed(96, i), l, 0, m if side == "left" else n, 0, l)
        it, _ = _item(A, phi, k, l, q, side, core, orth, kind=kind)
        items.append(it)
    h = corutv.Handle()
    try:
        b = corutv.Batch(items, handle=h)
        b.run()
        h.set_tracing(True)
        res = b.run()
        t = h.trace_read()
        h.set_tracing(False)
    finally:
        h.close()
    assert all(r.info.status == 0 for r in res)
    assert t.pass_launches > 0
    assert t.pass_kernel_launches == t.pass_launches
    assert 0.0 < t.pass_kernel_ms < t.pass_ms
