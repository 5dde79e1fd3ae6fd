"""Host logic of the decomposed cluster on CPU: splitter choice and top cells from
reduced counts, and the exchanges over two gloo ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from paper_2110_11658_b300 import decomp


def _counts_from_keys(keys):
    def fn(ranges):
        return np.array([np.count_nonzero((keys >= lo) & (keys < hi)) for lo, hi in ranges], dtype=np.int64)
    return fn


def _check_splitters(keys, bounds, threshold):
    keys = np.sort(keys)
    n = keys.size
    P = len(bounds) - 1
    for s, b in enumerate(bounds[1:-1], start=1):
        # every cell straddling the splitter holds more than the threshold
        for level in range(decomp.LEVELS):
            first, end = decomp.cell_bounds(level, b)
            if first == b:
                break
            inside = np.count_nonzero((keys >= first) & (keys < end))
            left = np.count_nonzero((keys >= first) & (keys < b))
            if 0 < left < inside:
                assert inside > threshold
        # and the split lies near the quantile
        assert abs(np.searchsorted(keys, b) - n * s // P) <= 8 * threshold


@pytest.mark.parametrize("kind,n,P", [("plummer", 20000, 2), ("plummer", 20000, 5), ("king", 30000, 3)])
def test_splitters_rule(kind, n, P):
    c = synth.make(kind, n, synth.BASE_SEED + P, masses="kroupa")
    keys = oracle.morton_keys(c.x, c.y, c.z).astype(np.uint64).astype(object)
    k64 = np.array([int(k) for k in keys], dtype=np.uint64)
    bounds = decomp.choose_splitters(n, P, 512, _counts_from_keys(k64))
    assert bounds[0] == 0 and bounds[-1] == decomp.KEY_END and all(a < b for a, b in zip(bounds, bounds[1:]))
    _check_splitters(k64, bounds[:], 512)
    tops = decomp.top_cells(bounds, _counts_from_keys(k64))
    for key, level in tops:
        first, end = decomp.cell_bounds(level, key)
        assert first == key and np.count_nonzero((k64 >= first) & (k64 < end)) > 512
    # the root straddles every splitter
    assert (0, 0) in tops


def test_splitters_refuse_a_split_root():
    with pytest.raises(ValueError):
        decomp.choose_splitters(100, 2, 512, lambda r: np.zeros(len(r), dtype=np.int64))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = decomp.TorchComm(dist)
        c = synth.plummer(20000, synth.BASE_SEED + 7, masses="kroupa")
        keys = oracle.morton_keys(c.x, c.y, c.z)
        mine = keys[rank::world]  # this rank's share of the particles
        def counts(ranges):  # noqa: E306
            loc = _counts_from_keys(mine)(ranges)
            return comm.allreduce([loc], "sum")[0]
        bounds = decomp.choose_splitters(c.n, world, 512, counts)
        tops = decomp.top_cells(bounds, counts)
        # exchange: each rank sends the others its keys that belong to them
        gid = np.arange(c.n)[rank::world]
        send = [[torch.from_numpy(gid[(mine >= bounds[d]) & (mine < bounds[d + 1])].astype(np.int64))
                 for d in range(world)]]
        got = np.sort(np.concatenate([t.numpy() for t in comm.alltoall(send)[0]]))
        q.put((rank, bounds, tops, got.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_and_exchange():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, b0, t0, g0), (r1, b1, t1, g1) = res
    assert b0 == b1 and t0 == t1  # both ranks take the same decisions
    c = synth.plummer(20000, synth.BASE_SEED + 7, masses="kroupa")
    keys = oracle.morton_keys(c.x, c.y, c.z)
    # the same splitters as from all keys at once, and every particle delivered to its rank
    assert b0 == decomp.choose_splitters(c.n, 2, 512, _counts_from_keys(keys))
    for r, got in ((0, g0), (1, g1)):
        want = np.nonzero((keys >= b0[r]) & (keys < b0[r + 1]))[0]
        assert got == want.tolist()
