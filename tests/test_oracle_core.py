"""Pins of the oracle's nearest-neighbour search and core quantities."""
import math

import numpy as np
import pytest

import oracle
import synth


def _np_knn(x, y, z, sample, k):
    idx = np.zeros((len(sample), k), np.int32)
    d2 = np.zeros((len(sample), k))
    j = np.arange(len(x))
    for t, i in enumerate(sample):
        dx, dy, dz = x - x[i], y - y[i], z - z[i]
        r2 = (dx * dx + dy * dy) + dz * dz  # the same FP64 operations
        r2[i] = np.inf
        o = np.lexsort((j, r2))[:k]
        idx[t], d2[t] = o, r2[o]
    return idx, d2


def test_knn_equals_sorting_brute_force_with_ties():
    # a lattice has many equal distances: ties go to the smaller index
    g = np.arange(6, dtype=float)
    x, y, z = (a.ravel() for a in np.meshgrid(g, g, g, indexing="ij"))
    rng = np.random.default_rng(3)
    sample = rng.choice(x.size, 40, replace=False).astype(np.int32)
    for k in (1, 6, 9):
        idx, d2 = oracle.knn(x, y, z, sample, k)
        ri, rd = _np_knn(x, y, z, sample, k)
        assert np.array_equal(idx, ri) and np.array_equal(d2, rd)
    c = synth.plummer(3000, 7)
    sample = rng.choice(c.n, 100, replace=False).astype(np.int32)
    idx, d2 = oracle.knn(c.x, c.y, c.z, sample, 6)
    ri, rd = _np_knn(c.x, c.y, c.z, sample, 6)
    assert np.array_equal(idx, ri) and np.array_equal(d2, rd)


def test_knn_with_fewer_candidates_than_k():
    x = np.array([0.0, 1.0, 3.0]); y = np.zeros(3); z = np.zeros(3)
    idx, d2 = oracle.knn(x, y, z, np.array([0], np.int32), 6)
    assert list(idx[0]) == [1, 2, -1, -1, -1, -1]
    assert d2[0, 0] == 1.0 and d2[0, 1] == 9.0 and np.all(np.isinf(d2[0, 2:]))


def test_density_of_an_octahedron_by_hand():
    # particle 0 at the origin, six neighbours at distance 1 on the axes, then far ones
    pts = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (5, 5, 5), (-6, 4, 3)]
    x, y, z = (np.array([p[d] for p in pts], float) for d in range(3))
    m = np.array([0.5, 1, 2, 3, 4, 5, 6, 7, 8], float)
    sample = np.array([0], np.int32)
    idx, d2 = oracle.knn(x, y, z, sample, 6)
    rho, q = oracle.core_quantities(x, y, z, m, sample, idx, d2)
    assert rho[0] == pytest.approx(3 * (1 + 2 + 3 + 4 + 5) / (4 * math.pi))
    assert np.allclose(q["centre"], 0.0) and q["r_core"] == 0.0 and q["n_core"] == 0


def test_density_estimator_is_unbiased_on_a_uniform_cube():
    rng = np.random.default_rng(11)
    n = 40000
    p = rng.random((3, n))
    m = np.full(n, 1.0 / n)  # density 1 in the unit cube
    inner = np.nonzero(np.all((p > 0.2) & (p < 0.8), axis=0))[0][:3000].astype(np.int32)
    idx, d2 = oracle.knn(p[0], p[1], p[2], inner, 6)
    rho, q = oracle.core_quantities(p[0], p[1], p[2], m, inner, idx, d2)
    assert np.mean(rho) == pytest.approx(1.0, rel=0.05)


def test_core_quantities_follow_their_definitions():
    c = synth.plummer(20000, 12)
    rng = np.random.default_rng(12)
    s = int(min(c.n, math.sqrt(5000 * c.n)))
    sample = rng.choice(c.n, s, replace=False).astype(np.int32)
    idx, d2 = oracle.knn(c.x, c.y, c.z, sample, 6)
    rho, q = oracle.core_quantities(c.x, c.y, c.z, c.m, sample, idx, d2)
    # recompute every quantity from its definition
    r_ = 3 * c.m[idx[:, :5]].sum(axis=1) / (4 * math.pi * np.sqrt(d2[:, 5]) ** 3)
    assert np.allclose(rho, r_, rtol=1e-13)
    P = np.stack([c.x[sample], c.y[sample], c.z[sample]], 1)
    cen = (rho[:, None] * P).sum(0) / rho.sum()
    assert np.allclose(q["centre"], cen, rtol=1e-11, atol=1e-14)
    rc = math.sqrt((rho ** 2 * ((P - cen) ** 2).sum(1)).sum() / (rho ** 2).sum())
    assert q["r_core"] == pytest.approx(rc, rel=1e-11)
    assert q["rho_core"] == pytest.approx((rho ** 2).sum() / rho.sum(), rel=1e-12)
    r2all = (c.x - q["centre"][0]) ** 2 + (c.y - q["centre"][1]) ** 2 + (c.z - q["centre"][2]) ** 2
    assert abs(q["n_core"] - int((r2all < q["r_core"] ** 2).sum())) <= 1
    # a Plummer sphere (a = 3 pi / 16, central density 3 / (4 pi a^3)): the density
    # centre sits at the origin and the core is of the order of a
    a = 3 * math.pi / 16
    assert np.linalg.norm(q["centre"]) < 0.1 * a
    assert 0.2 * a < q["r_core"] < 2 * a
    assert 0.2 < q["rho_core"] / (3 / (4 * math.pi * a ** 3)) < 2
