"""Serving with continuous batching (paper_2110_11658_b300/serve.py) on the GPU.

Each cluster's results must not depend on which other clusters shared its
batches: a mixed, overlapped run of many requests leaves every cluster in the
same state, bit for bit, as running the same steps one cluster at a time.
Results delivered through the arena (cluster-local neighbour rows,
accelerations) must equal the oracle's neighbour lists and a plain
single-cluster run."""
import numpy as np
import pytest
import torch

import oracle
import paper_2110_11658_b300 as p3t
import synth
from gpu_helpers import DEV, to_dev
from paper_2110_11658_b300.serve import Arena, Server, poisson_arrivals

pytestmark = pytest.mark.gpu

DT = 1.0 / 512


def _clusters():
    sizes = synth.log_uniform_sizes(10, 500, 20000, 77)
    cl = [synth.make("plummer" if k % 2 == 0 else "king", int(n), 300 + k, masses="kroupa", w0=7.0)
          for k, n in enumerate(sizes)]
    rows = []
    for c in cl:
        rc = synth.paper_run_params(c.n)["r_cut"]
        rows.append([0.5, 0.1 * rc, rc, rc])
    return cl, rows


def _arena_snapshot(ar):
    out = {k: v.cpu().numpy().copy() for k, v in ar.state.items()}
    out.update({"a%d" % i: a.cpu().numpy().copy() for i, a in enumerate(ar.acc)})
    out["offs"] = ar.nbr_offsets.cpu().numpy().copy()
    idx = ar.nbr_idx.cpu().numpy()
    offs = out["offs"]
    # compare only the filled part of each cluster's entry region
    out["idx"] = np.concatenate([idx[ar.ent_off[k]:ar.ent_off[k] + offs[ar.row_off[k] + ar.sizes[k]]]
                                 for k in range(ar.n_clusters)])
    return out


def test_mixed_batches_equal_one_cluster_at_a_time():
    torch.cuda.set_device(DEV)
    cl, rows = _clusters()
    steps = 3
    order = [k for _ in range(steps) for k in range(len(cl))]
    rng = np.random.default_rng(5)
    rng.shuffle(order)  # per-cluster order is all that matters
    arr = [(1e-4 * i, k) for i, k in enumerate(order)]

    ar_mix = Arena(cl, rows, device=DEV)
    big = max(ar_mix.sizes)
    srv = Server(ar_mix, n_slots=2, budget=int(2.5 * big), max_clusters=8, dt=DT)
    reqs = srv.run(arr)
    assert all(np.isfinite(r.t_done) for r in reqs)
    assert max(b[2] for b in srv.batches) > 1  # batches really mixed clusters
    mix = _arena_snapshot(ar_mix)
    srv.close()

    ar_one = Arena(cl, rows, device=DEV)
    one = Server(ar_one, n_slots=1, budget=big, max_clusters=1, dt=DT)
    one.run_serial(order)
    alone = _arena_snapshot(ar_one)
    one.close()
    for k in mix:
        assert np.array_equal(mix[k], alone[k]), k


def test_served_step_matches_oracle_neighbours_and_plain_run():
    torch.cuda.set_device(DEV)
    cl, rows = _clusters()
    ar = Arena(cl, rows, device=DEV)
    srv = Server(ar, n_slots=2, budget=int(2.5 * max(ar.sizes)), max_clusters=8, dt=DT)
    srv.run([(0.0, k) for k in range(len(cl))])
    for k, c in enumerate(cl):
        v = ar.cluster_view(k)
        offs = v["offsets"].cpu().numpy()
        idx = v["idx_base"][:int(offs[-1])].cpu().numpy()
        o2, i2 = oracle.neighbours_brute(c.x, c.y, c.z, rows[k][3])
        assert np.array_equal(offs, o2) and np.array_equal(idx, i2), k
        prm = p3t.Params(theta=rows[k][0], r_in=rows[k][1], r_out=rows[k][2], r_list=rows[k][3])
        ctx = p3t.Context(prm)
        ctx.build_tree(to_dev(c.x), to_dev(c.y), to_dev(c.z), to_dev(c.m))
        a = [torch.empty(c.n, dtype=torch.float32, device=DEV) for _ in range(3)]
        ctx.far_force(*a)
        ctx.check()
        for i in range(3):
            assert torch.equal(a[i], v["a"][i]), (k, i)
        vx = to_dev(c.vx) + 0.5 * DT * a[0].double()
        assert torch.equal(vx, v["vx"]), k
        ctx.close()
    srv.close()


def test_poisson_stream_serves_every_request():
    torch.cuda.set_device(DEV)
    cl, rows = _clusters()
    ar = Arena(cl, rows, device=DEV)
    srv = Server(ar, n_slots=2, budget=int(3 * max(ar.sizes)), max_clusters=16, dt=DT)
    reqs = srv.run(poisson_arrivals(2000.0, 300, len(cl), 9))
    assert all(r.t_done >= r.t_launch >= r.t_arrival for r in reqs)
    assert sum(b[2] for b in srv.batches) == 300
    srv.close()
