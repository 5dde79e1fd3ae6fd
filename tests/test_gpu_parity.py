"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Bit-exact: Morton keys, sort permutation, node topology, groups, FP64 moments
(COM, boxes, opening radii), per-group interaction counts, neighbour lists
and the kick.  Forces: the all-FP64 form within 1e-10 relative of the oracle
tree; the mixed form within median 1e-5 and 99th percentile 1e-4 (the
target accuracy of the distant-force path).
"""
import numpy as np
import pytest
import torch

import opening_cases
import oracle
import paper_2110_11658_b300 as p3t
import synth
from gpu_helpers import DEV, assert_tree_equal, rel_err, run_gpu, to_dev

pytestmark = pytest.mark.gpu

MIXED, FP64 = p3t.P3T_FP32_MIXED, p3t.P3T_FP64

CASES = [
    # id, kind, n, masses, theta, r_out, leaf, G
    ("plummer4096", "plummer", 4096, "equal", 0.5, 0.05, 16, 64),
    ("king20k_kroupa", "king", 20000, "kroupa", 0.4, 0.02, 8, 32),
    ("plummer3333_G128", "plummer", 3333, "kroupa", 0.7, 0.08, 16, 128),
    ("plummer257_leaf1", "plummer", 257, "equal", 0.3, 0.05, 1, 64),
    ("plummer33_G50", "plummer", 33, "equal", 0.5, 0.2, 4, 50),
]


def _case(kind, n, masses):
    return synth.make(kind, n, synth.BASE_SEED + n, masses=masses)


def _oracle(c, theta, r_out, leaf, G):
    return oracle.Tree(c.x, c.y, c.z, c.m, theta, r_out, leaf_cap=leaf, group_size=G)


@pytest.mark.parametrize("cid,kind,n,masses,theta,r_out,leaf,G", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
def test_tree_forces_counts_neighbours(cid, kind, n, masses, theta, r_out, leaf, G, precision):
    c = _case(kind, n, masses)
    r_in = 0.1 * r_out
    prm = p3t.Params(theta=theta, r_in=r_in, r_out=r_out, r_list=r_out, leaf_cap=leaf,
                     group_size=G, precision=precision)
    g = run_gpu(c, prm, kick_dt=1.0 / 256)
    t = _oracle(c, theta, r_out, leaf, G)
    ref = t.export()
    assert_tree_equal(g["tree"], ref, fp64_moments=precision == FP64)
    f = t.far(r_in)
    # identical interaction lists: per-group counts equal the oracle's
    assert np.array_equal(g["g_cells"], f["n_cell"])
    assert np.array_equal(g["g_parts"], f["n_part"])
    gc = ref["g_count"].astype(np.int64)
    assert g["n_cell"] == int((gc * f["n_cell"]).sum())
    assert g["n_part"] == int((gc * f["n_part"]).sum())
    e = rel_err(g["a"], f["a"])
    ep = np.abs(g["pot"] - f["pot"]) / np.abs(f["pot"])
    if precision == FP64:
        assert e.max() < 1e-10, e.max()
        assert ep.max() < 1e-12
    else:
        assert np.median(e) <= 1e-5 and np.percentile(e, 99) <= 1e-4, (np.median(e), np.percentile(e, 99))
        assert np.median(ep) <= 1e-6 and ep.max() < 1e-4
    # neighbour lists, bit-exact
    o2, i2 = oracle.neighbours_brute(c.x, c.y, c.z, r_out)
    assert np.array_equal(g["offs"], o2)
    assert np.array_equal(g["idx"], i2)
    # kick of Eq. 12 on the GPU's own accelerations, bit-exact
    v = oracle.kick(1.0 / 256, g["a"][:, 0], g["a"][:, 1], g["a"][:, 2], c.vx, c.vy, c.vz)
    assert np.array_equal(g["v"], np.stack(v, 1))


@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
def test_theta_zero_reproduces_direct_sum(precision):
    c = synth.plummer(512, 77, masses="kroupa")
    prm = p3t.Params(theta=0.0, r_in=0.005, r_out=0.05, r_list=0.05, leaf_cap=8, group_size=32,
                     precision=precision)
    g = run_gpu(c, prm, nbr=False)
    d = oracle.direct_split(c.x, c.y, c.z, c.m, 0.005, 0.05)
    e = rel_err(g["a"], d["far"])
    assert g["n_cell"] == 0 and g["n_part"] == 512 * 512
    assert e.max() < (1e-11 if precision == FP64 else 1e-5)


@pytest.mark.parametrize("r_list", [0.01, 0.05, 0.13])
def test_neighbour_radius_independent_of_r_out(r_list):
    c = synth.king(6000, 5, 7.0)
    prm = p3t.Params(theta=0.5, r_in=0.004, r_out=0.04, r_list=r_list, leaf_cap=16, group_size=64)
    g = run_gpu(c, prm, pot=False)
    o2, i2 = oracle.neighbours_brute(c.x, c.y, c.z, r_list)
    assert np.array_equal(g["offs"], o2) and np.array_equal(g["idx"], i2)
    assert (np.diff(o2) == 0).any() or r_list > 0.1  # empty rows occur and are legal


def test_quadrupole_off_matches_oracle_monopole():
    c = synth.plummer(4096, 3)
    prm = p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, quadrupole=0, precision=FP64, group_size=64)
    g = run_gpu(c, prm, nbr=False)
    f = _oracle(c, 0.5, 0.05, 16, 64).far(0.005, quadrupole=False)
    assert rel_err(g["a"], f["a"]).max() < 1e-10


def test_edge_cases_tiny_and_degenerate():
    rng = np.random.default_rng(4)
    cases = []
    # one particle: no force, no neighbours
    cases.append(synth.Cluster(*(np.array([0.3]) for _ in range(3)), np.array([1.0]),
                               *(np.zeros(1) for _ in range(3))))
    # two coincident particles: W(0) = 0 -> no far force; they are neighbours
    cases.append(synth.Cluster(np.array([0.1, 0.1]), np.array([0.2, 0.2]), np.array([0.3, 0.3]),
                               np.array([0.5, 0.5]), *(np.zeros(2) for _ in range(3))))
    # all particles at one point: side 0 -> 1, one level-21 leaf, chunked groups
    n = 300
    cases.append(synth.Cluster(np.full(n, -1.5), np.full(n, 2.0), np.full(n, 0.25),
                               np.full(n, 1.0 / n), *(np.zeros(n) for _ in range(3))))
    # a clump of duplicates inside a Plummer sphere, with some massless particles
    p = synth.plummer(2000, 9)
    p.x[:150] = p.x[0]
    p.y[:150] = p.y[0]
    p.z[:150] = p.z[0]
    p.m[rng.choice(2000, 100, replace=False)] = 0.0
    cases.append(p)
    for c in cases:
        for precision in (FP64, MIXED):
            prm = p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05, precision=precision,
                             group_size=32)
            g = run_gpu(c, prm)
            t = _oracle(c, 0.5, 0.05, 16, 32)
            ref = t.export()
            assert_tree_equal(g["tree"], ref, fp64_moments=precision == FP64)
            f = t.far(0.005)
            assert np.array_equal(g["g_cells"], f["n_cell"])
            assert np.array_equal(g["g_parts"], f["n_part"])
            scale = np.abs(f["a"]).max() + 1e-300
            assert np.abs(g["a"] - f["a"]).max() <= (1e-12 if precision == FP64 else 1e-5) * scale
            o2, i2 = oracle.neighbours_brute(c.x, c.y, c.z, 0.05)
            assert np.array_equal(g["offs"], o2) and np.array_equal(g["idx"], i2)


def test_repeatable_bitwise():
    c = synth.plummer(30000, 12, masses="kroupa")
    prm = p3t.Params(theta=0.4, r_in=0.004, r_out=0.04, r_list=0.04)
    a = run_gpu(c, prm, nbr=True)
    b = run_gpu(c, prm, nbr=True)
    assert np.array_equal(a["a"], b["a"]) and np.array_equal(a["pot"], b["pot"])
    assert np.array_equal(a["idx"], b["idx"])


@pytest.mark.parametrize("scale", [1e-8, 1e4])
def test_extreme_scales_switch_filters_off_or_on(scale):
    # at tiny scales the FP32 filters are switched off and every opening and
    # neighbour decision is taken in FP64; lists and counts must still match
    c = synth.plummer(3000, 31, masses="kroupa")
    c.x, c.y, c.z = c.x * scale, c.y * scale, c.z * scale
    r_out = 0.05 * scale
    prm = p3t.Params(theta=0.5, r_in=0.1 * r_out, r_out=r_out, r_list=0.8 * r_out, group_size=32)
    g = run_gpu(c, prm)
    t = _oracle(c, 0.5, r_out, 16, 32)
    assert_tree_equal(g["tree"], t.export(), fp64_moments=False)
    f = t.far(0.1 * r_out)
    assert np.array_equal(g["g_cells"], f["n_cell"]) and np.array_equal(g["g_parts"], f["n_part"])
    e = rel_err(g["a"], f["a"])
    assert np.median(e) <= 1e-5 and np.percentile(e, 99) <= 1e-4
    o2, i2 = oracle.neighbours_brute(c.x, c.y, c.z, 0.8 * r_out)
    assert np.array_equal(g["offs"], o2) and np.array_equal(g["idx"], i2)


def test_long_neighbour_rows_take_every_sort_path():
    # short rows (Plummer) and tight clumps whose rows fill every length class of
    # the row sort: [1, 4] (one thread a row), (4, 32], (32, 64], (64, 128] and
    # (128, 256], (256, 512], (512, 1024] (register networks, strided and
    # transposed), (1024, 2048] (shared memory) and > 2048 (global memory); every
    # row must equal the brute force
    p = synth.plummer(3000, 41)
    rng = np.random.default_rng(41)
    xs, ys, zs = [p.x], [p.y], [p.z]
    for n_c, centre in ((50, 2.5), (100, -2.5), (200, 3.0), (400, -3.0), (700, 2.0), (1500, 3.5),
                        (3000, -2.0)):
        q = rng.normal(size=(3, n_c)) * 0.002 + centre
        xs.append(q[0]), ys.append(q[1]), zs.append(q[2])
    x, y, z = np.concatenate(xs), np.concatenate(ys), np.concatenate(zs)
    n = x.size
    c = synth.Cluster(x, y, z, np.full(n, 1.0 / n), *(np.zeros(n) for _ in range(3)))
    g = run_gpu(c, p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05), pot=False)
    o2, i2 = oracle.neighbours_brute(x, y, z, 0.05)
    lens = np.diff(o2)
    for lo, hi in ((0, 1), (1, 4), (4, 32), (32, 64), (64, 128), (128, 256), (256, 512), (512, 1024),
                   (1024, 2048), (2048, n)):
        assert ((lens > lo) & (lens <= hi)).any(), (lo, hi)
    assert np.array_equal(g["offs"], o2) and np.array_equal(g["idx"], i2)


def test_row_mode_lists_and_fallback():
    # After one synchronous list of a tree that the far-force walk counted, the
    # following walks also write each neighbour into the context's row scratch and
    # the lists only sort those rows.  Each row's room comes from its particle's
    # last count (c + c/8 + 8).  A Plummer sphere plus a clump of 400 that is loose
    # (few neighbours) on the first steps and tight (399 each) on the last: those
    # rows overflow their room and come from the fill pass instead.  Every step's
    # lists equal the brute force, and the forces equal those of a context that
    # never enters row mode, bit for bit.
    p = synth.plummer(20000, 43)
    rng = np.random.default_rng(43)
    q = rng.normal(size=(3, 400))
    n = p.n + 400
    m = np.full(n, 1.0 / n)
    prm = p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05)
    ctx = p3t.Context(prm)
    a = [torch.empty(n, dtype=torch.float32, device=DEV) for _ in range(3)]
    offs = torch.empty(n + 1, dtype=torch.int64, device=DEV)
    idx = torch.empty(400 * 400 + 8 * n, dtype=torch.int32, device=DEV)
    for step, scale in enumerate((0.3, 0.3, 0.002, 0.002)):
        x, y, z = (np.concatenate([a_, b_]) for a_, b_ in zip((p.x, p.y, p.z), q * scale + 2.0))
        o2, i2 = oracle.neighbours_brute(x, y, z, 0.05)
        if scale < 0.01:
            assert np.diff(o2).max() == 399
        xd, yd, zd, md = to_dev(x), to_dev(y), to_dev(z), to_dev(m)
        ctx.build_tree(xd, yd, zd, md)
        ctx.far_force(*a)
        cap, valid = ctx.row_mode()
        if step == 0:
            assert cap == 0 and valid == 0
        else:
            assert cap > 0 and valid == 1
        tot = ctx.neighbours(offs, idx)
        assert tot == len(i2)
        assert np.array_equal(offs.cpu().numpy(), o2) and np.array_equal(idx[:tot].cpu().numpy(), i2)
    ctx2 = p3t.Context(prm)
    ctx2.build_tree(xd, yd, zd, md)
    b = [torch.empty(n, dtype=torch.float32, device=DEV) for _ in range(3)]
    ctx2.far_force(*b)
    ctx.check()
    ctx2.check()
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_row_mode_in_host_step():
    # p3t_step_host builds the lists before the far force, so its count pass
    # writes the rows from the second step on; lists (a clump's rows of 399
    # included) equal the brute force every step, accelerations and velocities
    # equal a first step (no row mode) of a fresh context
    p = synth.plummer(20000, 47)
    rng = np.random.default_rng(47)
    q = rng.normal(size=(3, 400)) * 0.002 - 2.0
    x, y, z = (np.concatenate([a, b]) for a, b in zip((p.x, p.y, p.z), q))
    n = x.size
    m = np.full(n, 1.0 / n)
    v = [np.concatenate([a, np.zeros(400)]) for a in (p.vx, p.vy, p.vz)]
    prm = p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05)
    o2, i2 = oracle.neighbours_brute(x, y, z, 0.05)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731

    def host_step(ctx):
        hv = [pin(a) for a in v]
        ha = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(3)]
        ho = torch.empty(n + 1, dtype=torch.int64).pin_memory()
        hi = torch.empty(2 * len(i2) + 64, dtype=torch.int32).pin_memory()
        tot = ctx.step_host(1.0 / 512, pin(x), pin(y), pin(z), pin(m), *hv, *ha, ho, hi)
        return tot, ho.numpy(), hi[:tot].numpy(), [t.numpy() for t in ha], [t.numpy() for t in hv]

    ref = host_step(p3t.Context(prm))
    ctx = p3t.Context(prm)
    for step in range(3):
        tot, offs, idx, acc, vel = host_step(ctx)
        cap, valid = ctx.row_mode()
        assert (valid == 1) == (step > 0) and cap > 0
        assert tot == len(i2) and np.array_equal(offs, o2) and np.array_equal(idx, i2)
        for u, w in zip(acc + vel, ref[3] + ref[4]):
            assert np.array_equal(u, w)


@pytest.mark.parametrize("case", opening_cases.CASES, ids=[c[0] for c in opening_cases.CASES])
@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
def test_opening_rule_decision_by_decision(case, precision):
    # the hand-built pairs that pin the oracle's opening rule one decision at a
    # time, several of them exactly on a threshold: the GPU's decisions (the
    # mixed form's FP32 filter falls back to FP64 inside its error band) give the
    # same per-group counts as the oracle and as the hand-worked table
    cid, theta, r_out, X, sx, sy, gy, opened, why = case
    x, y, z, m = opening_cases.particles(X, sx, sy, gy)
    c = synth.Cluster(x=x, y=y, z=z, m=m, vx=np.zeros_like(x), vy=np.zeros_like(x), vz=np.zeros_like(x))
    prm = p3t.Params(theta=theta, r_in=0.1 * r_out, r_out=r_out, r_list=r_out,
                     leaf_cap=opening_cases.LEAF_CAP, group_size=opening_cases.GROUP_SIZE,
                     precision=precision)
    g = run_gpu(c, prm, pot=False, nbr=False)
    t = oracle.Tree(x, y, z, m, theta, r_out, leaf_cap=opening_cases.LEAF_CAP,
                    group_size=opening_cases.GROUP_SIZE)
    f = t.far(0.1 * r_out)
    assert np.array_equal(g["g_cells"], f["n_cell"])
    assert np.array_equal(g["g_parts"], f["n_part"])
    grp = int(np.nonzero(g["tree"]["g_first"] == 0)[0][0])
    assert (int(g["g_cells"][grp]), int(g["g_parts"][grp])) == opening_cases.expected_counts(opened), why


@pytest.mark.parametrize("G", [64, 128])
@pytest.mark.parametrize("precision", [FP64, MIXED], ids=["fp64", "mixed"])
def test_threads_per_group_forms(G, precision):
    # G threads per group (the first warp walks, every warp evaluates its own 32
    # targets) evaluate the same tiles in the same order as one warp holding G/32
    # targets per lane: counts and lists bit for bit, and so are the mixed form's
    # forces (explicit FP32 intrinsics); the FP64 form's plain expressions may be
    # contracted into FMAs differently in the two kernels (1e-13); both against
    # the oracle's tree of the same G
    c = synth.make("king", 20000, synth.BASE_SEED + 5, masses="kroupa")
    base = dict(theta=0.4, r_in=0.002, r_out=0.02, r_list=0.02, leaf_cap=8, group_size=G, precision=precision)
    one = run_gpu(c, p3t.Params(threads_per_group=32, **base), kick_dt=1.0 / 256)
    many = run_gpu(c, p3t.Params(threads_per_group=G, **base), kick_dt=1.0 / 256)
    exact = ("g_cells", "g_parts", "offs", "idx") + (("a", "pot", "v") if precision == MIXED else ())
    for k in exact:
        assert np.array_equal(one[k], many[k]), k
    if precision == FP64:
        assert rel_err(many["a"], one["a"]).max() < 1e-13
        assert np.abs(many["pot"] - one["pot"]).max() < 1e-13 * np.abs(one["pot"]).max()
    assert one["n_cell"] == many["n_cell"] and one["n_part"] == many["n_part"]
    t = _oracle(c, 0.4, 0.02, 8, G)
    f = t.far(0.002)
    assert np.array_equal(many["g_cells"], f["n_cell"])
    assert np.array_equal(many["g_parts"], f["n_part"])
    e = rel_err(many["a"], f["a"])
    if precision == FP64:
        assert e.max() < 1e-10
    else:
        assert np.median(e) <= 1e-5 and np.percentile(e, 99) <= 1e-4
    o2, i2 = oracle.neighbours_brute(c.x, c.y, c.z, 0.02)
    assert np.array_equal(many["offs"], o2) and np.array_equal(many["idx"], i2)


@pytest.mark.parametrize("G", [64, 128])
def test_threads_per_group_row_mode(G):
    # with one target per thread the walk also writes the neighbour rows (row mode)
    # from the second step on; lists equal the brute force, forces the first step's
    c = synth.plummer(30000, synth.BASE_SEED + 6, masses="kroupa")
    prm = p3t.Params(theta=0.5, r_in=0.003, r_out=0.03, r_list=0.03, leaf_cap=16, group_size=G,
                     threads_per_group=G)
    ctx = p3t.Context(prm)
    d = [to_dev(getattr(c, k)) for k in "xyzm"]
    a = [torch.empty(c.n, dtype=torch.float32, device=DEV) for _ in range(3)]
    offs = torch.empty(c.n + 1, dtype=torch.int64, device=DEV)
    idx = torch.empty(64 * c.n, dtype=torch.int32, device=DEV)
    ctx.build_tree(*d)
    ctx.far_force(*a)
    ctx.neighbours(offs, idx)
    first = torch.stack(a, 1).double().cpu().numpy()
    o2, i2 = oracle.neighbours_brute(c.x, c.y, c.z, 0.03)
    for _ in range(2):
        ctx.build_tree(*d)
        ctx.far_force(*a)
        cap, valid = ctx.row_mode()
        assert cap > 0 and valid == 1
        tot = ctx.neighbours(offs, idx)
        ctx.check()
        assert np.array_equal(offs.cpu().numpy(), o2) and np.array_equal(idx[:tot].cpu().numpy(), i2)
        assert np.array_equal(torch.stack(a, 1).double().cpu().numpy(), first)
    ctx.close()


def test_cell_forms_agree():
    # The mixed walk evaluates cells in the r^-5 form when every cluster's r_out,
    # frame and mass keep it inside FP32, else in the r^-3 form.  Masses scaled by
    # 2^54 (total 1.8e16, past the 1e15 bound) select the r^-3 form; the scaling
    # is exact in both forms, so the two runs must give the same lists and forces
    # that agree to FP32 rounding, each within the oracle tolerance.
    c = synth.plummer(20000, 61, masses="kroupa")
    prm = p3t.Params(theta=0.4, r_in=0.004, r_out=0.04, r_list=0.04, group_size=32)
    fast = run_gpu(c, prm, pot=False)
    s = 2.0 ** 54
    heavy = synth.Cluster(c.x, c.y, c.z, c.m * s, c.vx, c.vy, c.vz)
    slow = run_gpu(heavy, prm, pot=False)
    assert np.array_equal(fast["g_cells"], slow["g_cells"]) and np.array_equal(fast["g_parts"], slow["g_parts"])
    assert np.array_equal(fast["offs"], slow["offs"]) and np.array_equal(fast["idx"], slow["idx"])
    a3 = slow["a"] / s
    e = rel_err(fast["a"], a3)
    assert np.median(e) < 1e-6 and e.max() < 1e-4, (np.median(e), e.max())
    assert not np.array_equal(fast["a"], a3)  # two different operation sequences ran
    f = _oracle(c, 0.4, 0.04, 16, 32).far(0.004)
    for a in (fast["a"], a3):
        err = rel_err(a, f["a"])
        assert np.median(err) <= 1e-5 and np.percentile(err, 99) <= 1e-4


@pytest.mark.parametrize("leaf", [2, 128, 129, 300])
def test_topology_flat_and_level_forms(leaf):
    """The topology is built flat (per-particle first and last levels, one scan) for
    leaf capacities up to 128 and level by level above: both give the oracle's tree
    node for node, with a clump of duplicates (level-21 leaves) in the mix."""
    c = synth.plummer(30000, 31, masses="kroupa")
    c.x[:400] = c.x[7]
    c.y[:400] = c.y[7]
    c.z[:400] = c.z[7]
    prm = p3t.Params(theta=0.5, r_in=0.003, r_out=0.03, r_list=0.03, leaf_cap=leaf, group_size=32)
    g = run_gpu(c, prm, pot=False, nbr=False)
    t = oracle.Tree(c.x, c.y, c.z, c.m, 0.5, 0.03, leaf_cap=leaf, group_size=32)
    assert_tree_equal(g["tree"], t.export(), fp64_moments=False)
    f = t.far(0.003)
    assert np.array_equal(g["g_cells"], f["n_cell"])
    assert np.array_equal(g["g_parts"], f["n_part"])
