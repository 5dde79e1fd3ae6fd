"""The flat topology's derivation, checked on the CPU against the oracle's tree.

The CUDA build numbers the canonical octree's nodes without a pass per level: particle i
(key order) starts the cells of levels s(i)+1 .. lam(i), where s(i) is the number of
levels its key shares with key i-1 (-1 at the start) and lam(i) = min(M(i)+1, 21) with
M(i) the largest number of levels shared by keys j and j+L over the windows [j, j+L]
that contain i (L = leaf capacity; a level-l cell holds more than L particles iff such a
window lies inside it).  Nodes are ordered by (level, first particle); node (l, i) is
split iff l < lam(i), its first child is (l+1, i), its count runs to the first key that
leaves its prefix, and its children are the next nodes of level l+1 that start inside it.
This module restates those steps in numpy (no GPU) and compares every node field with the
oracle's level-by-level build (Sec. 2.4's Barnes-Hut tree: split a node holding more than
leaf_cap particles, down to 21 levels).
"""
import numpy as np
import pytest

import oracle

LEVELS = 21


def shared_levels(a, b):
    """Levels (3 key bits each, below the unused top bit) that keys a and b share."""
    x = np.bitwise_xor(a, b).astype(np.uint64)
    out = np.full(x.shape, LEVELS, dtype=np.int64)
    nz = x != 0
    # index of the highest set bit; equal bits below bit 63 = 62 - msb
    msb = np.floor(np.log2(x[nz].astype(np.float64))).astype(np.int64)
    # float rounding can put a value just below 2^k at k: correct it exactly
    msb = np.where((np.uint64(1) << msb.astype(np.uint64)) > x[nz], msb - 1, msb)
    out[nz] = np.minimum((62 - msb) // 3, LEVELS)
    return out


def flat_topology(keys, L):
    n = len(keys)
    sh = np.full(n, -1, dtype=np.int64)
    if n > 1:
        sh[1:] = shared_levels(keys[:-1], keys[1:])
    w = np.full(n, -1, dtype=np.int64)
    if n > L:
        w[: n - L] = shared_levels(keys[: n - L], keys[L:])
    lam = np.zeros(n, dtype=np.int64)
    for i in range(n):
        j0, j1 = max(i - L, 0), min(i, n - 1 - L)
        m = w[j0 : j1 + 1].max() if j1 >= j0 else -1
        lam[i] = min(m + 1, LEVELS)
    nodes = sorted((l, i) for i in range(n) for l in range(sh[i] + 1, lam[i] + 1))
    ids = {nd: k for k, nd in enumerate(nodes)}
    level = np.array([l for l, _ in nodes])
    first = np.array([i for _, i in nodes])
    child = np.array([ids[(l + 1, i)] if l < lam[i] else -1 for l, i in nodes])
    count = np.zeros(len(nodes), dtype=np.int64)
    nchild = np.zeros(len(nodes), dtype=np.int64)
    for k, (l, i) in enumerate(nodes):
        end = n
        if l > 0:
            s = np.uint64(63 - 3 * l)
            p = keys[i] >> s
            end = i + 1
            while end < n and (keys[end] >> s) == p:
                end += 1
        count[k] = end - i
        if child[k] >= 0:
            c = child[k]
            while c < len(nodes) and level[c] == l + 1 and first[c] < end:
                c += 1
            nchild[k] = c - child[k]
    return dict(level=level, first=first, count=count, child=child, nchild=nchild)


@pytest.mark.parametrize("case", ["cubed_normal", "grid_duplicates", "uniform", "tiny"])
@pytest.mark.parametrize("L", [1, 3, 16])
def test_flat_topology_equals_level_by_level(case, L):
    rng = np.random.default_rng(hash((case, L)) % (2**32))
    n = {"cubed_normal": 1500, "grid_duplicates": 1200, "uniform": 1500, "tiny": 5}[case]
    if case == "cubed_normal":
        x = rng.standard_normal((n, 3)) ** 3  # a dense core and far outliers: deep cells
    elif case == "grid_duplicates":
        x = rng.integers(0, 4, (n, 3)).astype(float)  # many equal keys: level-21 leaves
    else:
        x = rng.random((n, 3))
    t = oracle.Tree(x[:, 0], x[:, 1], x[:, 2], np.ones(n), 0.5, 0.1, leaf_cap=L, group_size=16)
    ref = t.export()
    got = flat_topology(ref["keys"], L)
    for k in ("level", "first", "count", "child", "nchild"):
        assert np.array_equal(got[k], ref[k]), k


def test_shared_levels_definition():
    # keys equal above bit 3k+2 and different at it share exactly 20 - k levels
    a = np.array([0, 0, 0, (1 << 62)], dtype=np.uint64)
    b = np.array([0, 1, 1 << 60, 0], dtype=np.uint64)
    assert list(shared_levels(a, b)) == [21, 20, 0, 0]
