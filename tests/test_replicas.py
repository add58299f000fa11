"""The multi-GPU path of bench.py is replicas only (independent realizations
per rank, no data-path collective): its host bookkeeping -- disjoint seeds per
rank, the slowest rank's time via one all-reduce, whole-job throughput -- run
as two gloo ranks on CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=ws, init_method=f"tcp://127.0.0.1:{port}")
    import bench

    t, v = bench.aggregate(100.0 + 50.0 * rank, 2, ws, "cpu")
    q.put((rank, t, v, bench.replica_seeds(rank, ws, 3), bench.replica_seeds(rank, ws, 2, offset=10 ** 6)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_seed_disjointly():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, t, v, seeds, warm in res:
        assert t == 150.0                      # the slowest rank's time on every rank
        assert abs(v - 3 * 2 * 2 / 0.150) < 1e-9  # 12 solves in 150 ms
    assert not set(res[0][3]) & set(res[1][3])
    assert not set(res[0][4]) & set(res[1][4])
    assert res[0][3] == [0, 2, 4] and res[1][3] == [1, 3, 5]


def test_single_rank_needs_no_process_group():
    import bench

    t, v = bench.aggregate(250.0, 5, 1, "cpu")
    assert t == 250.0 and abs(v - 60.0) < 1e-12
    assert bench.replica_seeds(0, 1, 3) == [0, 1, 2]
