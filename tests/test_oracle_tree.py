"""Pins of the oracle's reference tree (Sec. 2.4) against independent constructions.

Keys are checked on a dyadic grid where every FP64 step is exact, the sort
against numpy's lexsort, the topology against an explicit recursion, the
moments against direct sums over each node's particles, the far force against
the direct sum at theta = 0 and against the multipole expansion of a
two-particle cell.
"""
import math

import numpy as np
import pytest

import opening_cases
import oracle
import synth

Q21 = 1 << 21


def spread_bits(q: int, lane: int) -> int:
    out = 0
    for k in range(21):
        out |= ((q >> k) & 1) << (3 * k + lane)
    return out


def test_interleave_by_hand():
    assert oracle.interleave(1, 0, 0) == 4
    assert oracle.interleave(0, 1, 0) == 2
    assert oracle.interleave(0, 0, 1) == 1
    assert oracle.interleave(2, 0, 0) == 32
    assert oracle.interleave(Q21 - 1, Q21 - 1, Q21 - 1) == (1 << 63) - 1
    assert oracle.interleave(Q21 - 1, 0, 0) == int("100" * 21, 2)


def test_keys_on_dyadic_grid():
    # cube [0,1]^3 fixed by two anchor points; cell centres (q + 1/2)/2^21 are exact
    rng = np.random.default_rng(7)
    q = rng.integers(0, Q21, size=(500, 3))
    pts = (q + 0.5) / Q21
    pts = np.vstack([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], pts])
    keys = oracle.morton_keys(pts[:, 0], pts[:, 1], pts[:, 2])
    assert keys[0] == 0
    assert int(keys[1]) == (1 << 63) - 1  # x = max maps to the clamped top cell
    for k, (a, b, c) in zip(keys[2:], q):
        assert int(k) == spread_bits(int(a), 2) | spread_bits(int(b), 1) | spread_bits(int(c), 0)
    cube = oracle.bounding_cube(pts[:, 0], pts[:, 1], pts[:, 2])
    assert list(cube) == [0.0, 0.0, 0.0, 1.0]


def test_degenerate_cube():
    # all particles at one point: side 1, all keys 0
    x = np.full(10, 0.25)
    assert list(oracle.bounding_cube(x, x, x)) == [0.25, 0.25, 0.25, 1.0]
    assert not oracle.morton_keys(x, x, x).any()


def _recursive_topology(keys, n, leaf_cap):
    """Explicit recursion over octants; returns nodes as (level, first, count) BFS-sorted."""
    nodes = []

    def rec(level, first, count):
        nodes.append((level, first, count))
        if count <= leaf_cap or level >= 21:
            return
        shift = 63 - 3 * (level + 1)
        digits = (keys[first:first + count] >> np.uint64(shift)) & np.uint64(7)
        for o in range(8):
            sel = np.nonzero(digits == o)[0]
            if sel.size:
                rec(level + 1, first + int(sel[0]), int(sel.size))

    rec(0, 0, n)
    # breadth-first: by level, then by first particle (= key prefix order)
    return sorted(nodes)


@pytest.mark.parametrize("kind,n,leaf", [("plummer", 3000, 16), ("plummer", 700, 1),
                                         ("king", 2000, 8)])
def test_sort_topology_moments(kind, n, leaf):
    c = synth.make(kind, n, synth.BASE_SEED + 11, masses="kroupa")
    t = oracle.Tree(c.x, c.y, c.z, c.m, theta=0.5, r_out=0.05, leaf_cap=leaf, group_size=64)
    d = t.export()
    keys = oracle.morton_keys(c.x, c.y, c.z)
    perm = np.lexsort((np.arange(n), keys))
    assert np.array_equal(d["perm"], perm)
    assert np.array_equal(d["keys"], keys[perm])
    ref = _recursive_topology(d["keys"], n, leaf)
    got = sorted(zip(d["level"].tolist(), d["first"].tolist(), d["count"].tolist()))
    assert got == ref
    assert list(zip(d["level"], d["first"], d["count"])) == [tuple(r) for r in ref]
    # children: contiguous, partition the parent's range in order
    for k in range(t.n_nodes):
        if d["nchild"][k]:
            ch = range(d["child"][k], d["child"][k] + d["nchild"][k])
            assert d["first"][ch[0]] == d["first"][k]
            assert sum(d["count"][j] for j in ch) == d["count"][k]
            for a, b in zip(ch, list(ch)[1:]):
                assert d["first"][b] == d["first"][a] + d["count"][a]
        else:
            assert d["count"][k] <= leaf or d["level"][k] == 21
    # moments against direct sums over each node's particles
    xs = np.stack([c.x, c.y, c.z], 1)[perm]
    ms = c.m[perm]
    for k in range(0, t.n_nodes, max(1, t.n_nodes // 300)):
        f, cnt = d["first"][k], d["count"][k]
        p, m = xs[f:f + cnt], ms[f:f + cnt]
        M = m.sum()
        com = (m[:, None] * p).sum(0) / M
        dd = p - com
        r2 = (dd ** 2).sum(1)
        Q = np.array([(m * (3 * dd[:, a] * dd[:, b] - (r2 if a == b else 0))).sum()
                      for a, b in [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]])
        assert d["M"][k] == pytest.approx(M, rel=1e-13)
        assert np.abs(d["com"][k] - com).max() < 1e-13 * (1 + np.abs(com).max())
        qs = (m * r2).sum() + 1e-300
        assert np.abs(d["Q"][k] - Q).max() < 1e-11 * qs
        assert abs(d["Q"][k][0] + d["Q"][k][3] + d["Q"][k][5]) < 1e-12 * qs  # traceless
        assert np.array_equal(d["lo"][k], p.min(0)) and np.array_equal(d["hi"][k], p.max(0))
        ext = p.max(0) - p.min(0)
        delta = np.linalg.norm(0.5 * (p.max(0) + p.min(0)) - com)
        assert d["ropen2"][k] == pytest.approx((ext.max() / 0.5 + delta) ** 2, rel=1e-13)


def test_groups_partition_and_rule():
    c = synth.plummer(5000, synth.BASE_SEED + 5)
    for g in (8, 32, 64, 128):
        t = oracle.Tree(c.x, c.y, c.z, c.m, 0.5, 0.05, leaf_cap=16, group_size=g)
        d = t.export()
        f, n = d["g_first"], d["g_count"]
        assert f[0] == 0 and np.array_equal(f[1:], (f + n)[:-1]) and f[-1] + n[-1] == 5000
        assert n.max() <= g
        # rebuild the rule by recursion: chunks of g inside nodes of <= 16 g
        # particles whose parent holds more (or big leaves)
        expect = []

        def rec(k):
            cnt = d["count"][k]
            if cnt <= 16 * g or d["nchild"][k] == 0:
                for s0 in range(0, cnt, g):
                    expect.append((d["first"][k] + s0, min(g, cnt - s0)))
                return
            for j in range(d["child"][k], d["child"][k] + d["nchild"][k]):
                rec(j)

        rec(0)
        assert sorted(expect) == list(zip(f.tolist(), n.tolist()))
        xs = np.stack([c.x, c.y, c.z], 1)[d["perm"]]
        for i in range(len(f)):
            p = xs[f[i]:f[i] + n[i]]
            assert np.array_equal(d["g_lo"][i], p.min(0)) and np.array_equal(d["g_hi"][i], p.max(0))


def test_big_leaf_is_chunked():
    # 1201 coincident particles at 0.5 plus 0, 0.25 (octant 0) and 0.75, 1
    # (octant 7): with G = 64 the level-21 leaf of 1201 > 16 G is cut into 18
    # chunks of 64 and one of 49; the two 2-particle branches are groups
    x = np.concatenate([np.full(1200, 0.5), np.linspace(0, 1, 5)])
    m = np.full(x.size, 1.0 / x.size)
    t = oracle.Tree(x, x, x, m, 0.5, 0.01, leaf_cap=16, group_size=64)
    d = t.export()
    assert d["level"].max() == 21
    leaf21 = np.nonzero((d["level"] == 21) & (d["count"] > 64))[0]
    assert d["count"][leaf21].tolist() == [1201]
    assert sorted(d["g_count"].tolist()) == sorted([2, 2, 49] + [64] * 18)
    f0 = d["first"][leaf21[0]]
    chunks = [(f0 + 64 * k, 64) for k in range(18)] + [(f0 + 1152, 49)]
    assert set(chunks) <= set(zip(d["g_first"].tolist(), d["g_count"].tolist()))


def test_theta_zero_is_direct_sum():
    for n, seed in [(512, 1), (300, 2), (97, 3)]:
        c = synth.plummer(n, seed, masses="kroupa")
        d = oracle.direct_split(c.x, c.y, c.z, c.m, 0.005, 0.05)
        for g in (32, 64):
            t = oracle.Tree(c.x, c.y, c.z, c.m, 0.0, 0.05, leaf_cap=8, group_size=g)
            f = t.far(0.005)
            scale = np.abs(d["far"]).max()
            assert np.abs(f["a"] - d["far"]).max() < 1e-13 * scale
            assert np.abs(f["pot"] - d["pot"]).max() < 1e-13 * np.abs(d["pot"]).max()
            assert f["n_cell"].sum() == 0
            assert np.array_equal(f["n_part"], np.full(t.n_groups, n))


def _rel_err(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def test_error_falls_with_theta_and_quadrupole_helps():
    c = synth.plummer(4096, synth.BASE_SEED, masses="kroupa")
    d = oracle.direct_split(c.x, c.y, c.z, c.m, 0.005, 0.05)
    med = {}
    for q in (True, False):
        for th in (0.7, 0.5, 0.3):
            t = oracle.Tree(c.x, c.y, c.z, c.m, th, 0.05, leaf_cap=16, group_size=64)
            e = _rel_err(t.far(0.005, quadrupole=q)["a"], d["far"])
            med[q, th] = (np.median(e), np.percentile(e, 99))
    for q in (True, False):
        assert med[q, 0.7][0] > med[q, 0.5][0] > med[q, 0.3][0]
        assert med[q, 0.7][1] > med[q, 0.5][1] > med[q, 0.3][1]
    for th in (0.7, 0.5, 0.3):
        assert med[True, th][0] < 0.5 * med[False, th][0]
    assert med[True, 0.5][0] < 1e-3


def test_two_particle_cell_multipole():
    # a cell of two masses seen from a distant group: monopole error ~ (s/r)^2,
    # quadrupole error ~ (s/r)^3, both along the exact expansion
    errs_q, errs_m = [], []
    for dist in (2.0, 4.0, 8.0):
        x = np.array([0.0, 0.013, dist])
        y = np.array([0.0, 0.007, 0.3])
        z = np.array([0.0, -0.004, 0.1])
        m = np.array([0.6, 0.4, 1e-12])
        t = oracle.Tree(x, y, z, m, theta=1.0, r_out=1e-3, leaf_cap=2, group_size=1)
        exact = oracle.direct_split(x, y, z, m, 1e-5, 1e-4, targets=[2])["far"][0]
        fq = t.far(1e-5, quadrupole=True)
        fm = t.far(1e-5, quadrupole=False)
        assert fq["n_cell"].sum() >= 1
        errs_q.append(np.linalg.norm(fq["a"][2] - exact) / np.linalg.norm(exact))
        errs_m.append(np.linalg.norm(fm["a"][2] - exact) / np.linalg.norm(exact))
    for a, b in zip(errs_m, errs_m[1:]):
        assert a / b == pytest.approx(4.0, rel=0.1)
    for a, b in zip(errs_q, errs_q[1:]):
        assert a / b == pytest.approx(8.0, rel=0.15)
    assert all(q < m for q, m in zip(errs_q, errs_m))


def test_accepted_cells_are_beyond_r_out():
    # with theta = 0.5 the far force of isolated particles from accepted cells is
    # unweighted; every P-P pair closer than r_out is inside an opened leaf, so
    # tree far + direct near reproduces the full force to the multipole error
    c = synth.plummer(4096, synth.BASE_SEED)
    t = oracle.Tree(c.x, c.y, c.z, c.m, 0.3, 0.05, leaf_cap=16, group_size=64)
    f = t.far(0.005)
    d = oracle.direct_split(c.x, c.y, c.z, c.m, 0.005, 0.05)
    e = _rel_err(f["a"] + d["near"], d["full"])
    assert np.median(e) < 1e-4


@pytest.mark.parametrize("r_list", [0.02, 0.05, 0.11])
def test_tree_neighbours_equal_brute_force(r_list):
    c = synth.king(3000, synth.BASE_SEED + 3, 7.0)
    t = oracle.Tree(c.x, c.y, c.z, c.m, 0.5, 0.05, leaf_cap=16, group_size=64)
    counts, offs, idx = t.neighbours(r_list)
    o2, i2 = oracle.neighbours_brute(c.x, c.y, c.z, r_list)
    assert np.array_equal(counts, np.diff(o2))
    assert np.array_equal(offs, o2) and np.array_equal(idx, i2)
    # a selection of groups gives the same rows
    sel = np.arange(0, t.n_groups, 3)
    cs, os_, is_ = t.neighbours(r_list, groups=sel)
    rows = np.nonzero(cs >= 0)[0]
    for i in rows[::17]:
        assert np.array_equal(is_[os_[i]:os_[i + 1]], i2[o2[i]:o2[i + 1]])


def test_sampled_groups_match_full_walk():
    c = synth.plummer(4096, synth.BASE_SEED + 9, masses="kroupa")
    t = oracle.Tree(c.x, c.y, c.z, c.m, 0.4, 0.05, leaf_cap=16, group_size=64)
    full = t.far(0.005)
    sel = np.array([0, 5, t.n_groups - 1])
    part = t.far(0.005, groups=sel)
    rows = ~np.isnan(part["a"][:, 0])
    assert rows.sum() == sum(t.export()["g_count"][sel])
    assert np.array_equal(part["a"][rows], full["a"][rows])
    assert np.array_equal(part["n_cell"], full["n_cell"][sel])
    assert math.isfinite(full["a"].sum())


@pytest.mark.parametrize("case", opening_cases.CASES, ids=[c[0] for c in opening_cases.CASES])
def test_opening_rule_decision_by_decision(case):
    # one hand-built group/cell pair per case, on one side of a threshold of the
    # opening rule or exactly on it; the expected decision is worked out by hand
    # in the case table, with the mistake that would flip it
    cid, theta, r_out, X, sx, sy, gy, opened, why = case
    x, y, z, m = opening_cases.particles(X, sx, sy, gy)
    t = oracle.Tree(x, y, z, m, theta, r_out, leaf_cap=opening_cases.LEAF_CAP,
                    group_size=opening_cases.GROUP_SIZE)
    d = t.export()
    # the layout the table assumes: the root's children are the group's leaf,
    # the cell's leaf and the ballast's branch, in that order
    kids = list(range(d["child"][0], d["child"][0] + d["nchild"][0]))
    assert [d["count"][k] for k in kids] == [2, 2, opening_cases.BALLAST]
    assert d["nchild"][kids[0]] == 0 and d["nchild"][kids[1]] == 0
    assert d["perm"][:4].tolist() == [0, 1, 2, 3]
    g = int(np.nonzero(d["g_first"] == 0)[0][0])
    assert d["g_count"][g] == 2
    f = t.far(0.1 * r_out, groups=[g])
    assert (int(f["n_cell"][0]), int(f["n_part"][0])) == opening_cases.expected_counts(opened), why
