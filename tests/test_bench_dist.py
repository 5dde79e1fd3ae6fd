"""Host logic of bench.py's multi-rank (replica) path on two gloo ranks, on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "P3T_BENCH_BACKEND": "gloo"})
    import bench
    r, local, w = bench.dist_init()
    bench.dist_barrier(w)
    t = bench.dist_max(1.0 + r, w)          # the slowest rank sets the time
    n = bench.dist_sum(1000.0 * (r + 1), w)  # particles of all replicas
    out.put((r, w, t, n))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 2.0, 3000.0), (1, 2, 2.0, 3000.0)]


def test_single_rank_is_identity():
    import bench
    assert bench.dist_max(3.5, 1) == 3.5 and bench.dist_sum(7.0, 1) == 7.0
