"""Sampled 6-nearest-neighbour search and core quantities on the GPU against the
oracle (p3t_sample_knn6, the tree search, and p3t_sample_knn6_brute, the
brute-force search; p3t_core_quantities)."""
import math

import numpy as np
import pytest
import torch

import bench
import oracle
import paper_2110_11658_b300 as p3t
import synth
from gpu_helpers import DEV, to_dev

pytestmark = pytest.mark.gpu


def _run(x, y, z, m, sample, brute=False, leaf_cap=16):
    ctx = p3t.Context(p3t.Params(leaf_cap=leaf_cap))
    d = [to_dev(a) for a in (x, y, z, m)]
    ctx.build_tree(*d)
    sm = torch.from_numpy(np.ascontiguousarray(sample, dtype=np.int32)).to(DEV)
    idx, d2 = ctx.sample_knn6(sm, brute=brute)
    rho, q = ctx.core_quantities(*d, sm, idx, d2)
    if len(x) < 7:  # no 6th neighbour: every density is 0
        assert np.all(rho.cpu().numpy() == 0)
    ctx.check()
    out = idx.cpu().numpy(), d2.cpu().numpy(), rho.cpu().numpy(), q
    ctx.close()
    return out


def _sample(n, seed):
    s = int(min(n, math.sqrt(5000 * n)))
    return np.random.default_rng(seed).choice(n, s, replace=False).astype(np.int32)


@pytest.mark.parametrize("brute", [False, True])
def test_knn_and_core_equal_oracle_plummer(brute):
    c = synth.plummer(50000, 71, masses="kroupa")
    sample = _sample(c.n, 71)
    gi, gd, grho, gq = _run(c.x, c.y, c.z, c.m, sample, brute)
    oi, od = oracle.knn(c.x, c.y, c.z, sample, 6)
    assert np.array_equal(gi, oi) and np.array_equal(gd, od)  # unique result, bit for bit
    orho, oq = oracle.core_quantities(c.x, c.y, c.z, c.m, sample, oi, od)
    assert np.allclose(grho, orho, rtol=1e-13, atol=0)
    assert np.allclose(gq["centre"], oq["centre"], rtol=1e-11, atol=1e-14)
    assert gq["r_core"] == pytest.approx(oq["r_core"], rel=1e-11)
    assert gq["rho_core"] == pytest.approx(oq["rho_core"], rel=1e-12)
    cen, rc = gq["centre"], gq["r_core"]
    r2 = ((c.x - cen[0]) * (c.x - cen[0]) + (c.y - cen[1]) * (c.y - cen[1])) + (c.z - cen[2]) * (c.z - cen[2])
    assert gq["n_core"] == int((r2 < rc * rc).sum())  # the count for the GPU's own centre
    assert abs(gq["n_core"] - oq["n_core"]) <= 1


@pytest.mark.parametrize("brute", [False, True])
def test_knn_ties_duplicates_and_short_lists(brute):
    g = np.arange(7, dtype=float)
    x, y, z = (a.ravel() for a in np.meshgrid(g, g, g, indexing="ij"))
    x = np.concatenate([x, x[:20]]); y = np.concatenate([y, y[:20]]); z = np.concatenate([z, z[:20]])
    m = np.full(x.size, 1.0 / x.size)
    sample = np.random.default_rng(72).choice(x.size, 120, replace=False).astype(np.int32)
    gi, gd, _, _ = _run(x, y, z, m, sample, brute)
    oi, od = oracle.knn(x, y, z, sample, 6)
    assert np.array_equal(gi, oi) and np.array_equal(gd, od)
    assert (gd == 0).any()  # coincident duplicates are nearest neighbours at distance 0
    # fewer than six other particles: -1 / inf padding
    x5 = np.array([0.0, 1.0, 2.5, 4.0, 9.0]); z5 = np.zeros(5)
    gi, gd, _, _ = _run(x5, z5, z5, np.full(5, 0.2), np.array([0, 4], np.int32), brute)
    oi, od = oracle.knn(x5, z5, z5, np.array([0, 4], np.int32), 6)
    assert np.array_equal(gi, oi) and np.array_equal(gd, od)
    assert list(gi[0]) == [1, 2, 3, 4, -1, -1]


def test_errors():
    c = synth.plummer(3000, 73)
    ctx = p3t.Context(p3t.Params())
    sm = torch.tensor([0, 5, 9], dtype=torch.int32, device=DEV)
    with pytest.raises(p3t.P3TError) as e:
        ctx.sample_knn6(sm, n=c.n)
    assert e.value.code == p3t.P3T_ERR_ORDER
    d = [to_dev(getattr(c, k)) for k in "xyzm"]
    ctx.build_tree(*d)
    bad = torch.tensor([0, c.n + 5, 9], dtype=torch.int32, device=DEV)
    ctx.sample_knn6(bad)
    assert ctx.status() == p3t.P3T_ERR_INVALID_INPUT
    seg = torch.tensor([0, 1000, c.n], dtype=torch.int64, device=DEV)
    ctx.build_tree_batch(seg, *d)
    with pytest.raises(p3t.P3TError) as e:
        ctx.sample_knn6(sm)  # several clusters
    assert e.value.code == p3t.P3T_ERR_ORDER
    ctx.close()


@pytest.mark.parametrize("brute", [False, True])
def test_fullsize_knn_on_a_subsample(brute):
    c, _ = bench.workload(bench.N_DEFAULT, 20211022)
    sample = np.random.default_rng(74).choice(c.n, 2000, replace=False).astype(np.int32)
    gi, gd, _, _ = _run(c.x, c.y, c.z, c.m, sample, brute)
    oi, od = oracle.knn(c.x, c.y, c.z, sample, 6)
    assert np.array_equal(gi, oi) and np.array_equal(gd, od)


def test_tree_knn_in_clumps_and_big_leaves():
    # tight clumps (key-order neighbours far from the sixth nearest at the clump
    # edges), duplicated points beyond the leaf capacity (leaves at the deepest
    # level) and a small leaf capacity: the tree search equals the oracle
    rng = np.random.default_rng(75)
    parts = [rng.normal(size=(3, 3000)) * 0.3]
    for centre in (4.0, -4.0, 9.0):
        parts.append(rng.normal(size=(3, 200)) * 1e-3 + centre)
    parts.append(np.repeat(np.array([[1.5], [1.5], [1.5]]), 40, axis=1))
    x, y, z = np.concatenate(parts, axis=1)
    m = np.full(x.size, 1.0 / x.size)
    sample = rng.choice(x.size, 600, replace=False).astype(np.int32)
    oi, od = oracle.knn(x, y, z, sample, 6)
    for leaf_cap in (2, 16):
        gi, gd, _, _ = _run(x, y, z, m, sample, leaf_cap=leaf_cap)
        assert np.array_equal(gi, oi) and np.array_equal(gd, od), leaf_cap
