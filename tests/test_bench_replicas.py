"""The multi-process replica logic of bench.py on CPU (gloo, world size 2): every rank
runs its own replicas, the barrier holds both, and the whole-job rate is the units of all
ranks over the slowest rank's time -- the same number on every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    # rank r took 100 (r + 1) ms for 3 steps
    value, ms = bench.replica_rate(3, 100.0 * (rank + 1), w)
    bench.barrier(w)
    dist.destroy_process_group()
    q.put((rank, value, ms))


def test_replica_rate_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, value, ms in res:
        assert ms == 200.0                      # the slowest rank's time
        assert abs(value - 2 * 3 / 0.2) < 1e-9  # 6 steps over 0.2 s


def test_replica_rate_single_process():
    import bench
    assert bench.replica_rate(5, 250.0, 1) == (20.0, 250.0)
