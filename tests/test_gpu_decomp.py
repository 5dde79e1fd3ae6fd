"""One cluster over several ranks, all ranks on one GPU (LocalComm).

Each rank builds its part of the tree, exports its locally essential trees and
joins the others'; its groups then walk the global tree.  Checked against the
oracle's tree of the whole cluster: the ranks' groups, in rank order, are the
oracle's groups with identical per-group interaction counts; forces within the
mixed form's tolerance (the all-FP64 form within 1e-10); neighbour rows of
global indices equal to the brute force bit for bit; and the forces equal to a
single-rank build of the whole cluster.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2110_11658_b300 as p3t
import synth
from gpu_helpers import DEV, rel_err, run_gpu, to_dev
from paper_2110_11658_b300 import decomp

pytestmark = pytest.mark.gpu

MIXED, FP64 = p3t.P3T_FP32_MIXED, p3t.P3T_FP64


def _run(c, prm, n_ranks, seed=0):
    rng = np.random.default_rng(seed)
    owner = rng.integers(0, n_ranks, size=c.n)  # an arbitrary first distribution
    comm = decomp.LocalComm(n_ranks)
    parts = []
    for r in range(n_ranks):
        sel = np.nonzero(owner == r)[0]
        ctx = p3t.Context(prm)
        ctx.set_debug(True)
        d = lambda a: to_dev(a[sel])  # noqa: E731
        parts.append(decomp.RankPart(ctx, d(c.x), d(c.y), d(c.z), d(c.m), d(c.vx), d(c.vy), d(c.vz),
                                     torch.from_numpy(sel.astype(np.int64)).to(DEV)))
    decomp.decompose(comm, parts, prm)
    out = []
    for p in parts:
        n = p.x.numel()
        a = [torch.empty(n, dtype=p.ctx.acc_dtype, device=DEV) for _ in range(3)]
        p.ctx.far_force(*a)
        offs = torch.empty(n + 1, dtype=torch.int64, device=DEV)
        idx = torch.empty(max(1, 64 * n), dtype=torch.int32, device=DEV)
        tot = p.ctx.neighbours(offs, idx)
        gc, gp = p.ctx.group_counts()
        p.ctx.check()
        out.append({"gid": p.gid.cpu().numpy(), "a": torch.stack(a, 1).double().cpu().numpy(),
                    "offs": offs.cpu().numpy(), "idx": idx[:tot].cpu().numpy(), "g_cells": gc.cpu().numpy(),
                    "g_parts": gp.cpu().numpy(), "info": p.info})
        p.ctx.close()
    return out


@pytest.mark.parametrize("kind,n,n_ranks,precision", [
    ("plummer", 30000, 2, MIXED), ("plummer", 30000, 3, MIXED), ("king", 20000, 2, FP64),
    ("king", 40000, 4, MIXED)], ids=["plummer30k_2", "plummer30k_3", "king20k_2_fp64", "king40k_4"])
def test_decomposed_step_equals_the_global_tree(kind, n, n_ranks, precision):
    c = synth.make(kind, n, synth.BASE_SEED + n + n_ranks, masses="kroupa")
    r_out = 0.03 if kind == "plummer" else 0.015
    prm = p3t.Params(theta=0.45, r_in=0.1 * r_out, r_out=r_out, r_list=r_out, leaf_cap=8, group_size=32,
                     precision=precision)
    res = _run(c, prm, n_ranks)
    assert all(r["info"]["top_cells"] > 0 for r in res)
    t = oracle.Tree(c.x, c.y, c.z, c.m, prm.theta, r_out, leaf_cap=8, group_size=32)
    f = t.far(prm.r_in)
    # the ranks' groups in rank order are the oracle's groups, with the same lists
    assert np.array_equal(np.concatenate([r["g_cells"] for r in res]), f["n_cell"])
    assert np.array_equal(np.concatenate([r["g_parts"] for r in res]), f["n_part"])
    gid = np.concatenate([r["gid"] for r in res])
    assert np.array_equal(np.sort(gid), np.arange(c.n))
    a = np.empty((c.n, 3))
    a[gid] = np.concatenate([r["a"] for r in res])
    e = rel_err(a, f["a"])
    if precision == FP64:
        assert e.max() < 1e-10, e.max()
    else:
        assert np.median(e) <= 1e-5 and np.percentile(e, 99) <= 1e-4, (np.median(e), np.percentile(e, 99))
    # neighbour rows of global indices, bit for bit
    o2, i2 = oracle.neighbours_brute(c.x, c.y, c.z, r_out)
    for r in res:
        for k, g in enumerate(r["gid"]):
            assert np.array_equal(r["idx"][r["offs"][k]:r["offs"][k + 1]], i2[o2[g]:o2[g + 1]]), g
    # and the same forces as one build of the whole cluster on one rank
    one = run_gpu(c, prm, pot=False, nbr=False)
    assert rel_err(a, one["a"]).max() < (1e-12 if precision == FP64 else 1e-5)


def test_splitters_at_cell_edges_and_balanced():
    c = synth.plummer(50000, synth.BASE_SEED + 1, masses="kroupa")
    prm = p3t.Params(theta=0.5, r_in=0.003, r_out=0.03, r_list=0.03, leaf_cap=16, group_size=32)
    res = _run(c, prm, 4, seed=3)
    counts = [len(r["gid"]) for r in res]
    assert sum(counts) == c.n
    # each rank near N / P: off by less than the largest cell a splitter may not enter
    assert max(abs(k - c.n / 4) for k in counts) <= 16 * 32 * 8
    keys = oracle.morton_keys(c.x, c.y, c.z)
    b = res[0]["info"]["bounds"]
    for r, rr in enumerate(res):
        kr = keys[rr["gid"]]
        assert kr.min() >= b[r] and (r == 3 or kr.max() < b[r + 1])
