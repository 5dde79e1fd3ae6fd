"""Parity of the 64-cluster ensemble at its full size, in the form the benchmark times.

64 clusters, alternately Plummer and King W0 = 5, N log-uniform in [1e4, 5e5]
(7.8e6 particles), equal masses, theta = 0.4, per-cluster r_out = the paper's
r_cut (Eqs. 21-22), r_in = 0.1 r_out, r_list = r_out, mixed precision, at the tuned
launch shape (G = 32, one warp per group, tile 64, leaf_cap 16).  As in the
benchmark, one synchronous list call sizes the row scratch, then the whole step is
captured into a CUDA graph (batched build, row-mode walk, lists, kick, drift) and
launched.  Against the oracle's tree of every cluster: the groups bit for bit,
every neighbour row bit for bit, and for 24 seeded groups per cluster the
interaction counts exactly and the forces within the mixed form's tolerance.
"""
import numpy as np
import pytest
import torch

import bench
import oracle
import paper_2110_11658_b300 as p3t
import synth
from gpu_helpers import DEV, rel_err

pytestmark = pytest.mark.gpu

SAMPLED_GROUPS = 24


def test_ensemble64_graph_step_against_oracle():
    cl = synth.ensemble(bench.ENS_CLUSTERS, bench.ENS_N_LO, bench.ENS_N_HI, 20211022, masses="equal", w0=5.0)
    allc, segn = synth.concat(cl)
    n = allc.n
    rows = bench.ensemble_params([c.n for c in cl])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)  # noqa: E731
    st = {k: t(getattr(allc, k)) for k in ("x", "y", "z", "m", "vx", "vy", "vz")}
    seg = t(segn)
    cprm = torch.tensor(rows, dtype=torch.float64, device=DEV)
    shape = bench.ENS_TUNED
    prm = p3t.Params(theta=bench.ENS_THETA, r_in=rows[0][1], r_out=rows[0][2], r_list=rows[0][3],
                     leaf_cap=shape["leaf_cap"], group_size=shape["group_size"], tile=shape["tile"],
                     threads_per_group=shape["threads_per_group"], precision=p3t.P3T_FP32_MIXED)
    a = [torch.empty(n, dtype=torch.float32, device=DEV) for _ in range(3)]
    offs = torch.empty(n + 1, dtype=torch.int64, device=DEV)
    idx = torch.empty(16 * n, dtype=torch.int32, device=DEV)
    tot = torch.zeros(1, dtype=torch.int64, device=DEV)
    ctx = p3t.Context(prm)
    ctx.set_debug(True)
    ctx.build_tree_batch(seg, st["x"], st["y"], st["z"], st["m"], cluster_params=cprm)
    ctx.far_force(*a)
    ctx.neighbours(offs, idx)
    g = ctx.capture_step(st["x"], st["y"], st["z"], st["m"], *a, seg_offsets=seg, cluster_params=cprm,
                         vx=st["vx"], vy=st["vy"], vz=st["vz"], kick_dt=bench.DT, drift_dt=bench.DT,
                         offsets=offs, idx=idx, total=tot)
    g.launch()  # the step of the positions it starts from (the drift comes last)
    ctx.check()
    cap, valid = ctx.row_mode()
    assert cap > 0 and valid == 1  # the captured walk wrote the neighbour rows
    ab = torch.stack(a, 1).double().cpu().numpy()
    ob = offs.cpu().numpy()
    ib = idx[: int(tot.item())].cpu().numpy()
    gc, gp = (v.cpu().numpy() for v in ctx.group_counts())
    tree = {k: v.cpu().numpy() for k, v in ctx.export_tree().items()}
    g.close()
    ctx.close()

    rng = np.random.default_rng(20211022)
    errs = []
    for k, c in enumerate(cl):
        s0, s1 = int(segn[k]), int(segn[k + 1])
        _, r_in, r_out, r_list = rows[k]
        ref = oracle.Tree(c.x, c.y, c.z, c.m, bench.ENS_THETA, r_out, leaf_cap=shape["leaf_cap"],
                          group_size=shape["group_size"])
        rx = ref.export()
        # this cluster's groups in the batched tree: the same groups, in the same order
        mine = np.nonzero((tree["g_first"] >= s0) & (tree["g_first"] < s1))[0]
        assert np.array_equal(tree["g_first"][mine] - s0, rx["g_first"]), k
        assert np.array_equal(tree["g_count"][mine], rx["g_count"]), k
        # every neighbour row of the cluster, by cluster-local original index
        _, ro, ri = ref.neighbours(r_list)
        assert np.array_equal(ob[s0:s1 + 1] - ob[s0], ro), k
        assert np.array_equal(ib[ob[s0]:ob[s1]] - s0, ri), k
        # sampled groups: counts exactly, forces within tolerance
        sel = np.sort(rng.choice(ref.n_groups, size=min(SAMPLED_GROUPS, ref.n_groups), replace=False))
        f = ref.far(r_in, groups=sel)
        assert np.array_equal(gc[mine[sel]], f["n_cell"]), k
        assert np.array_equal(gp[mine[sel]], f["n_part"]), k
        tg = np.nonzero(~np.isnan(f["a"][:, 0]))[0]
        errs.append(rel_err(ab[s0 + tg], f["a"][tg]))
    e = np.concatenate(errs)
    assert e.size > 64 * 200
    assert np.median(e) <= 1e-5 and np.percentile(e, 99) <= 1e-4
