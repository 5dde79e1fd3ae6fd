"""Ensemble form: one batched build of independent clusters of uneven size.

Each cluster's result from the batch must equal, bit for bit, the result of a
build of that cluster alone (per-cluster cubes, frames and roots), and match
the oracle's tree of that cluster."""
import numpy as np
import pytest
import torch

import oracle
import paper_2110_11658_b300 as p3t
import synth
from gpu_helpers import DEV, run_gpu, to_dev

pytestmark = pytest.mark.gpu


def _ensemble():
    specs = [("plummer", 3000, "equal"), ("king", 1, "equal"), ("plummer", 33, "kroupa"),
             ("king", 4096, "kroupa"), ("plummer", 2, "equal"), ("king", 777, "equal"),
             ("plummer", 5000, "kroupa")]
    cl = []
    for k, (kind, n, masses) in enumerate(specs):
        if n <= 2:
            rng = np.random.default_rng(k)
            p = rng.normal(size=(3, n)) * 0.1 + 3.0 * k
            cl.append(synth.Cluster(p[0], p[1], p[2], np.full(n, 1.0 / n), *(np.zeros(n) for _ in range(3))))
        else:
            c = synth.make(kind, n, 100 + k, masses=masses, w0=5.0)
            c.x = c.x + 5.0 * k  # clusters far apart and of different sizes
            cl.append(c)
    return cl


def _concat(cl):
    cat = lambda a: np.concatenate([getattr(c, a) for c in cl])  # noqa: E731
    seg = np.zeros(len(cl) + 1, np.int64)
    np.cumsum([c.n for c in cl], out=seg[1:])
    return synth.Cluster(*(cat(a) for a in ("x", "y", "z", "m", "vx", "vy", "vz"))), seg


@pytest.mark.parametrize("shape", [(32, 32), (64, 64), (128, 128)], ids=["G32", "G64x64thr", "G128x128thr"])
@pytest.mark.parametrize("precision", [p3t.P3T_FP32_MIXED, p3t.P3T_FP64], ids=["mixed", "fp64"])
def test_batch_equals_each_cluster_alone(precision, shape):
    # every launch shape the autotuner searches: G and threads per group
    G, tpg = shape
    cl = _ensemble()
    all_, seg = _concat(cl)
    prm = p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05, group_size=G, threads_per_group=tpg,
                     precision=precision)
    ctx = p3t.Context(prm)
    x, y, z, m = to_dev(all_.x), to_dev(all_.y), to_dev(all_.z), to_dev(all_.m)
    segd = torch.from_numpy(seg).to(DEV)
    ctx.build_tree_batch(segd, x, y, z, m)
    dt = ctx.acc_dtype
    n = all_.n
    a = [torch.empty(n, dtype=dt, device=DEV) for _ in range(3)]
    pot = torch.empty(n, dtype=torch.float64, device=DEV)
    ctx.far_force(*a, pot=pot)
    offs = torch.empty(n + 1, dtype=torch.int64, device=DEV)
    idx = torch.empty(50 * n, dtype=torch.int32, device=DEV)
    tot = ctx.neighbours(offs, idx)
    v = [to_dev(all_.vx), to_dev(all_.vy), to_dev(all_.vz)]
    ctx.kick(1.0 / 256, *a, *v)
    ctx.check()
    ab = torch.stack(a, 1).double().cpu().numpy()
    pb = pot.cpu().numpy()
    ob, ib = offs.cpu().numpy(), idx[:tot].cpu().numpy()
    vb = torch.stack(v, 1).cpu().numpy()
    info = ctx.tree_info()
    assert info["n"] == n
    for k, c in enumerate(cl):
        s0, s1 = seg[k], seg[k + 1]
        g = run_gpu(c, prm, kick_dt=1.0 / 256)
        assert np.array_equal(ab[s0:s1], g["a"])  # bit-identical
        assert np.array_equal(pb[s0:s1], g["pot"])
        assert np.array_equal(vb[s0:s1], g["v"])
        rows_b = ob[s0:s1 + 1] - ob[s0]
        assert np.array_equal(rows_b, g["offs"])
        assert np.array_equal(ib[ob[s0]:ob[s1]] - s0, g["idx"])
        t = oracle.Tree(c.x, c.y, c.z, c.m, 0.5, 0.05, leaf_cap=16, group_size=G)
        f = t.far(0.005)
        assert np.array_equal(g["g_cells"], f["n_cell"])
    assert tot == ob[-1]


def test_batch_rejects_bad_offsets():
    c = synth.plummer(1000, 3)
    ctx = p3t.Context(p3t.Params())
    bad = torch.tensor([0, 600, 500, 1000], dtype=torch.int64, device=DEV)  # not increasing
    ctx.build_tree_batch(bad, to_dev(c.x), to_dev(c.y), to_dev(c.z), to_dev(c.m))
    assert ctx.status() == p3t.P3T_ERR_INVALID_INPUT
    good = torch.tensor([0, 500, 1000], dtype=torch.int64, device=DEV)
    ctx.build_tree_batch(good, to_dev(c.x), to_dev(c.y), to_dev(c.z), to_dev(c.m))
    a = [torch.empty(1000, dtype=torch.float32, device=DEV) for _ in range(3)]
    ctx.far_force(*a)
    ctx.check()


@pytest.mark.parametrize("precision", [p3t.P3T_FP32_MIXED, p3t.P3T_FP64], ids=["mixed", "fp64"])
def test_batch_with_per_cluster_parameters(precision):
    # radii by the paper's rule per cluster size (Eqs. 20-25); one cluster lists
    # neighbours beyond r_out (counted by the count pass, not the walk) and one
    # asks for no neighbours at all
    cl = _ensemble()
    all_, seg = _concat(cl)
    rows = []
    for k, c in enumerate(cl):
        rc = synth.paper_run_params(max(c.n, 64))["r_cut"]
        theta = (0.3, 0.5, 0.7)[k % 3]
        r_list = rc if k not in (3, 5) else (1.5 * rc if k == 3 else 0.0)
        rows.append([theta, 0.1 * rc, rc, r_list])
    cprm = np.array(rows, dtype=np.float64)
    prm = p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05, group_size=32, precision=precision)
    ctx = p3t.Context(prm)
    n = all_.n
    ctx.build_tree_batch(torch.from_numpy(seg).to(DEV), to_dev(all_.x), to_dev(all_.y), to_dev(all_.z),
                         to_dev(all_.m), cluster_params=torch.from_numpy(cprm).to(DEV))
    a = [torch.empty(n, dtype=ctx.acc_dtype, device=DEV) for _ in range(3)]
    ctx.far_force(*a)
    offs = torch.empty(n + 1, dtype=torch.int64, device=DEV)
    idx = torch.empty(50 * n, dtype=torch.int32, device=DEV)
    tot = ctx.neighbours(offs, idx)
    ctx.check()
    ab = torch.stack(a, 1).double().cpu().numpy()
    ob, ib = offs.cpu().numpy(), idx[:tot].cpu().numpy()
    for k, c in enumerate(cl):
        th, ri, ro, rl = cprm[k]
        s0, s1 = seg[k], seg[k + 1]
        g = run_gpu(c, p3t.Params(theta=th, r_in=ri, r_out=ro, r_list=rl, group_size=32, precision=precision))
        assert np.array_equal(ab[s0:s1], g["a"])
        assert np.array_equal(ob[s0:s1 + 1] - ob[s0], g["offs"])
        assert np.array_equal(ib[ob[s0]:ob[s1]] - s0, g["idx"])
        o2, i2 = oracle.neighbours_brute(c.x, c.y, c.z, rl)
        assert np.array_equal(g["offs"], o2) and np.array_equal(g["idx"], i2)
    bad = cprm.copy()
    bad[2, 1] = bad[2, 2] * 2  # r_in > r_out
    ctx.build_tree_batch(torch.from_numpy(seg).to(DEV), to_dev(all_.x), to_dev(all_.y), to_dev(all_.z),
                         to_dev(all_.m), cluster_params=torch.from_numpy(bad).to(DEV))
    assert ctx.status() == p3t.P3T_ERR_INVALID_INPUT


def test_batch_row_mode_over_steps():
    # the same per-cluster batch stepped three times on one context: from the
    # second step the walk writes the rows (a cluster beyond r_out through the
    # shell ranges, one without neighbours); every step's lists equal each
    # cluster's brute force
    cl = _ensemble()
    all_, seg = _concat(cl)
    rows = []
    for k, c in enumerate(cl):
        rc = synth.paper_run_params(max(c.n, 64))["r_cut"]
        r_list = rc if k not in (3, 5) else (1.5 * rc if k == 3 else 0.0)
        rows.append([(0.3, 0.5, 0.7)[k % 3], 0.1 * rc, rc, r_list])
    cprm = np.array(rows, dtype=np.float64)
    prm = p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05, group_size=32)
    ctx = p3t.Context(prm)
    n = all_.n
    args = (torch.from_numpy(seg).to(DEV), to_dev(all_.x), to_dev(all_.y), to_dev(all_.z), to_dev(all_.m))
    a = [torch.empty(n, dtype=ctx.acc_dtype, device=DEV) for _ in range(3)]
    offs = torch.empty(n + 1, dtype=torch.int64, device=DEV)
    idx = torch.empty(50 * n, dtype=torch.int32, device=DEV)
    ref = [oracle.neighbours_brute(c.x, c.y, c.z, cprm[k, 3]) for k, c in enumerate(cl)]
    for step in range(3):
        ctx.build_tree_batch(*args, cluster_params=torch.from_numpy(cprm).to(DEV))
        ctx.far_force(*a)
        assert ctx.row_mode()[1] == (1 if step > 0 else 0)
        tot = ctx.neighbours(offs, idx)
        ctx.check()
        ob, ib = offs.cpu().numpy(), idx[:tot].cpu().numpy()
        for k, (o2, i2) in enumerate(ref):
            s0, s1 = seg[k], seg[k + 1]
            assert np.array_equal(ob[s0:s1 + 1] - ob[s0], o2)
            assert np.array_equal(ib[ob[s0]:ob[s1]] - s0, i2)


def test_batch_with_a_cluster_outside_the_r5_range():
    # One cluster whose mass (scaled by 2^54, past 1e15) puts it outside the r^-5 cell
    # term's FP32 range makes the whole batch take the r^-3 term: the other cluster's
    # lists stay bit-identical to its build alone (r^-5), its forces agree to FP32
    # rounding, and both clusters match the oracle.
    a_c = synth.plummer(3000, 71, masses="kroupa")
    b_c = synth.plummer(2000, 72, masses="kroupa")
    s = 2.0 ** 54
    b_c = synth.Cluster(b_c.x + 10.0, b_c.y, b_c.z, b_c.m * s, b_c.vx, b_c.vy, b_c.vz)
    all_, seg = _concat([a_c, b_c])
    prm = p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05, group_size=32)
    ctx = p3t.Context(prm)
    ctx.build_tree_batch(torch.from_numpy(seg).to(DEV), to_dev(all_.x), to_dev(all_.y), to_dev(all_.z),
                         to_dev(all_.m))
    n = all_.n
    a = [torch.empty(n, dtype=torch.float32, device=DEV) for _ in range(3)]
    ctx.far_force(*a)
    offs = torch.empty(n + 1, dtype=torch.int64, device=DEV)
    idx = torch.empty(50 * n, dtype=torch.int32, device=DEV)
    tot = ctx.neighbours(offs, idx)
    ctx.check()
    ab = torch.stack(a, 1).double().cpu().numpy()
    ob, ib = offs.cpu().numpy(), idx[:tot].cpu().numpy()
    alone = run_gpu(a_c, prm, pot=False)
    s0, s1 = seg[0], seg[1]
    assert np.array_equal(ob[s0:s1 + 1] - ob[s0], alone["offs"])
    assert np.array_equal(ib[ob[s0]:ob[s1]], alone["idx"])
    e = np.linalg.norm(ab[s0:s1] - alone["a"], axis=1) / np.linalg.norm(alone["a"], axis=1)
    assert np.median(e) < 1e-6 and e.max() < 1e-4
    for k, (c, scale) in enumerate(((a_c, 1.0), (b_c, s))):
        t = oracle.Tree(c.x, c.y, c.z, c.m, 0.5, 0.05, leaf_cap=16, group_size=32)
        ref = t.far(0.005)["a"]
        got = ab[seg[k]:seg[k + 1]]
        err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert np.median(err) <= 1e-5 and np.percentile(err, 99) <= 1e-4, (k, np.median(err), np.percentile(err, 99))


@pytest.mark.parametrize("leaf", [1, 128])
def test_batch_flat_topology_leaf_caps(leaf):
    """The flat topology of a batched build at both ends of its window (leaf capacity 1
    and 128), with a cluster of coincident points (one level-21 leaf): each cluster's
    forces equal its build alone bit for bit, and its walk counts the oracle's."""
    cl = _ensemble()[:6]
    n0 = 300
    cl.append(synth.Cluster(np.full(n0, 40.0), np.full(n0, -2.0), np.full(n0, 0.5), np.full(n0, 1.0 / n0),
                            *(np.zeros(n0) for _ in range(3))))
    all_, seg = _concat(cl)
    prm = p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05, leaf_cap=leaf, group_size=32)
    ctx = p3t.Context(prm)
    x, y, z, m = to_dev(all_.x), to_dev(all_.y), to_dev(all_.z), to_dev(all_.m)
    ctx.build_tree_batch(torch.from_numpy(seg).to(DEV), x, y, z, m)
    n = all_.n
    a = [torch.empty(n, dtype=ctx.acc_dtype, device=DEV) for _ in range(3)]
    ctx.far_force(*a)
    ctx.check()
    ab = torch.stack(a, 1).double().cpu().numpy()
    for k, c in enumerate(cl):
        s0, s1 = seg[k], seg[k + 1]
        g = run_gpu(c, prm, pot=False, nbr=False)
        assert np.array_equal(ab[s0:s1], g["a"])
        t = oracle.Tree(c.x, c.y, c.z, c.m, 0.5, 0.05, leaf_cap=leaf, group_size=32)
        f = t.far(0.005)
        assert np.array_equal(g["g_cells"], f["n_cell"])
        assert np.array_equal(g["g_parts"], f["n_part"])
