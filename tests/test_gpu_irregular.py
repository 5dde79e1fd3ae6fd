"""Irregular force and jerk over the neighbour rows (p3t_irregular) against the
oracle (Eqs. 1, 2, 7), on the rows the GPU neighbour pass produced."""
import numpy as np
import pytest
import torch

import oracle
import paper_2110_11658_b300 as p3t
import synth
from gpu_helpers import DEV, row_mass_over_r2, to_dev

pytestmark = pytest.mark.gpu

R_IN, R_OUT = 0.005, 0.05


def _cluster(n=20000, seed=61, s=0.35):
    c = synth.plummer(n, seed, masses="kroupa")
    c.x, c.y, c.z = c.x * s, c.y * s, c.z * s
    return c


def _gpu(c, prm, shift=None, seg=None, cprm=None):
    """Build, neighbour rows, irregular force on (optionally drifted) states."""
    ctx = p3t.Context(prm)
    d = {k: to_dev(getattr(c, k)) for k in ("x", "y", "z", "m", "vx", "vy", "vz")}
    if seg is None:
        ctx.build_tree(d["x"], d["y"], d["z"], d["m"])
    else:
        ctx.build_tree_batch(torch.from_numpy(seg).to(DEV), d["x"], d["y"], d["z"], d["m"],
                             cluster_params=torch.from_numpy(cprm).to(DEV))
    offs = torch.empty(c.n + 1, dtype=torch.int64, device=DEV)
    idx = torch.empty(200 * c.n, dtype=torch.int32, device=DEV)
    tot = ctx.neighbours(offs, idx)
    if shift is not None:  # predicted positions: the rows stay those of the build
        for q, v in zip("xyz", ("vx", "vy", "vz")):
            d[q] = d[q] + shift * d[v]
    f, j = ctx.irregular(offs, idx, d["x"], d["y"], d["z"], d["m"], d["vx"], d["vy"], d["vz"])
    ctx.check()
    out = {"f": f.T.cpu().numpy(), "j": j.T.cpu().numpy(), "offs": offs.cpu().numpy(),
           "idx": idx[:tot].cpu().numpy(), "pos": [d[q].cpu().numpy() for q in "xyz"]}
    ctx.close()
    return out


def _unweighted(c, g, r_out=R_OUT):
    x, y, z = g["pos"]
    return row_mass_over_r2(x, y, z, c.m, g["offs"], g["idx"], r_out)


def _oracle(c, g, r_in=R_IN, r_out=R_OUT):
    x, y, z = g["pos"]
    return oracle.irregular(x, y, z, c.m, c.vx, c.vy, c.vz, r_in, r_out, g["offs"], g["idx"], scales=True)


@pytest.mark.parametrize("shift", [None, 1e-3], ids=["built", "predicted"])
def test_fp64_form_equals_oracle(shift):
    c = _cluster()
    g = _gpu(c, p3t.Params(theta=0.5, r_in=R_IN, r_out=R_OUT, r_list=R_OUT, precision=p3t.P3T_FP64), shift)
    f, j, sf, sj = _oracle(c, g)
    assert (np.diff(g["offs"]) > 0).mean() > 0.8  # most particles have neighbours
    # same operations per pair; only the order of the row's sum differs
    assert np.all(np.abs(g["f"] - f).max(axis=1) <= 1e-13 * sf)
    assert np.all(np.abs(g["j"] - j).max(axis=1) <= 1e-13 * sj)


def test_mixed_form_within_fp32_error_of_oracle():
    c = _cluster()
    g = _gpu(c, p3t.Params(theta=0.5, r_in=R_IN, r_out=R_OUT, r_list=R_OUT), 1e-3)
    f, j, sf, sj = _oracle(c, g)
    # FP32 pair arithmetic: relative 1e-5 of the term magnitudes, plus an absolute
    # FP32 rounding of K (1e-7) times the unweighted row scale
    su = _unweighted(c, g)
    ef = np.abs(g["f"] - f).max(axis=1) / np.maximum(sf + 1e-2 * su, 1e-300)
    ej = np.abs(g["j"] - j).max(axis=1) / np.where(sj > 0, sj, 1)
    assert ef.max() <= 1e-5, ef.max()
    assert np.median(ef) <= 1e-6 and np.median(ej) <= 1e-6
    big = sj > 1e-3 * np.median(sj[sj > 0])
    assert ej[big].max() <= 1e-4, ej[big].max()
    rel = np.linalg.norm(g["f"] - f, axis=1) / np.maximum(np.linalg.norm(f, axis=1), 1e-300)
    ok = np.linalg.norm(f, axis=1) > 1e-3 * sf
    assert np.median(rel[ok]) <= 1e-5


def test_per_cluster_radii_after_batch_build():
    cl = [_cluster(3000, 62 + k, s) for k, s in enumerate((0.3, 0.5, 0.8))]
    allc, seg = synth.concat(cl)
    rows = np.array([[0.5, 0.1 * ro, ro, ro] for ro in (0.04, 0.06, 0.09)])
    g = _gpu(allc, p3t.Params(precision=p3t.P3T_FP64), seg=seg, cprm=rows)
    for k, c in enumerate(cl):
        s0, s1 = seg[k], seg[k + 1]
        ro, ri = rows[k, 2], rows[k, 1]
        offs = g["offs"][s0:s1 + 1] - g["offs"][s0]
        idx = g["idx"][g["offs"][s0]:g["offs"][s1]] - s0
        f, j, sf, sj = oracle.irregular(c.x, c.y, c.z, c.m, c.vx, c.vy, c.vz, ri, ro, offs, idx, scales=True)
        assert np.all(np.abs(g["f"][s0:s1] - f).max(axis=1) <= 1e-13 * sf)
        assert np.all(np.abs(g["j"][s0:s1] - j).max(axis=1) <= 1e-13 * sj)


def test_errors_order_and_bad_index():
    c = _cluster(2000, 63)
    ctx = p3t.Context(p3t.Params())
    d = {k: to_dev(getattr(c, k)) for k in ("x", "y", "z", "m", "vx", "vy", "vz")}
    offs = torch.zeros(c.n + 1, dtype=torch.int64, device=DEV)
    idx = torch.zeros(4, dtype=torch.int32, device=DEV)
    with pytest.raises(p3t.P3TError) as e:
        ctx.irregular(offs, idx, *(d[k] for k in ("x", "y", "z", "m", "vx", "vy", "vz")))
    assert e.value.code == p3t.P3T_ERR_ORDER
    ctx.build_tree(d["x"], d["y"], d["z"], d["m"])
    offs[1:] = 1  # row 0 = [index n] (out of range)
    idx[0] = c.n
    ctx.irregular(offs, idx, *(d[k] for k in ("x", "y", "z", "m", "vx", "vy", "vz")))
    assert ctx.status() == p3t.P3T_ERR_INVALID_INPUT
    ctx.close()
