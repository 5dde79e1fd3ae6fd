"""Neighbour lists with a buffer radius r_list = r_out + r_buff (Eq. 20).

The walk counts the neighbours beyond r_out through neighbour-only ranges; the
far force must not depend on r_list, and lists built at one regular step must
hold every pair that comes within r_out during the step, for pairs whose
relative displacement stays within r_buff (the buffer's purpose)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2110_11658_b300 as p3t
import synth
from gpu_helpers import DEV, rel_err, run_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("factor", [1.3, 2.0])
def test_far_force_independent_of_list_radius(factor):
    c = synth.plummer(20000, 81, masses="kroupa")
    c.x, c.y, c.z = c.x * 0.4, c.y * 0.4, c.z * 0.4
    base = dict(theta=0.5, r_in=0.004, r_out=0.04, group_size=32)
    a = run_gpu(c, p3t.Params(r_list=0.04, **base))
    b = run_gpu(c, p3t.Params(r_list=0.04 * factor, **base))
    # the same interaction lists (bit-exact counts per group); the massless shell
    # sources share the particle tiles, so the FP32 sums may round in another order
    for k in ("g_cells", "g_parts"):
        assert np.array_equal(a[k], b[k]), k
    assert a["n_cell"] == b["n_cell"] and a["n_part"] == b["n_part"]
    e = rel_err(b["a"], a["a"])
    assert e.max() < 1e-5 and np.median(e) < 1e-6, (e.max(), np.median(e))
    assert np.allclose(b["pot"], a["pot"], rtol=1e-6)
    for g, r in ((a, 0.04), (b, 0.04 * factor)):
        o, i = oracle.neighbours_brute(c.x, c.y, c.z, r)
        assert np.array_equal(g["offs"], o) and np.array_equal(g["idx"], i)


def test_buffered_lists_cover_a_regular_step():
    n = 50000
    c = synth.plummer(n, 82)
    pr = synth.paper_run_params(n)
    r_out, r_buff, dt = pr["r_cut"], pr["r_buff"], pr["dt_reg"]
    ctx = p3t.Context(p3t.Params(theta=0.4, r_in=0.1 * r_out, r_out=r_out, r_list=r_out + r_buff))
    ctx.build_tree(*(to_dev(getattr(c, k)) for k in "xyzm"))
    offs = torch.empty(n + 1, dtype=torch.int64, device=DEV)
    idx = torch.empty(64 * n, dtype=torch.int32, device=DEV)
    tot = ctx.neighbours(offs, idx)
    ctx.check()
    offs, idx = offs.cpu().numpy(), idx[:tot].cpu().numpy()
    o0, i0 = oracle.neighbours_brute(c.x, c.y, c.z, r_out + r_buff)
    assert np.array_equal(offs, o0) and np.array_equal(idx, i0)
    # one regular step of straight-line motion, then every pair inside r_out
    x1, y1, z1 = c.x + dt * c.vx, c.y + dt * c.vy, c.z + dt * c.vz
    o1, i1 = oracle.neighbours_brute(x1, y1, z1, r_out)
    old = set()
    for i in range(n):
        for j in idx[offs[i]:offs[i + 1]]:
            old.add((i, int(j)))
    missed_slow, missed, pairs = 0, 0, 0
    for i in range(n):
        for j in i1[o1[i]:o1[i + 1]]:
            pairs += 1
            if (i, int(j)) in old:
                continue
            missed += 1
            dv = np.array([c.vx[j] - c.vx[i], c.vy[j] - c.vy[i], c.vz[j] - c.vz[i]])
            if np.linalg.norm(dv) * dt <= r_buff:
                missed_slow += 1
    assert pairs > 1000
    assert missed_slow == 0  # guaranteed by the triangle inequality
    assert missed <= 0.01 * pairs  # the buffer covers nearly every pair (3 sigma)
