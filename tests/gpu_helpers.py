"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2110_11658_b300 as p3t

DEV = torch.device("cuda", 0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def run_gpu(c, prm: p3t.Params, pot=True, nbr=True, debug=True, kick_dt=None):
    """Build + far force (+ neighbours, + kick) on the GPU; everything back as numpy."""
    ctx = p3t.Context(prm)
    ctx.set_debug(debug)
    x, y, z, m = to_dev(c.x), to_dev(c.y), to_dev(c.z), to_dev(c.m)
    ctx.build_tree(x, y, z, m)
    dt = ctx.acc_dtype
    a = [torch.full((c.n,), float("nan"), dtype=dt, device=DEV) for _ in range(3)]
    ph = torch.full((c.n,), float("nan"), dtype=torch.float64, device=DEV) if pot else None
    nc = torch.zeros(1, dtype=torch.int64, device=DEV)
    np_ = torch.zeros(1, dtype=torch.int64, device=DEV)
    ctx.far_force(*a, pot=ph, n_cell=nc, n_part=np_)
    out = {"a": torch.stack(a, 1).double().cpu().numpy(), "n_cell": int(nc.item()),
           "n_part": int(np_.item())}
    if pot:
        out["pot"] = ph.cpu().numpy()
    ctx.check()
    out["tree"] = {k: v.cpu().numpy() for k, v in ctx.export_tree().items()}
    out["tree"]["keys"] = out["tree"]["keys"].view(np.uint64)
    if debug:
        gc, gp = ctx.group_counts()
        out["g_cells"], out["g_parts"] = gc.cpu().numpy(), gp.cpu().numpy()
    if nbr:
        offs = torch.empty(c.n + 1, dtype=torch.int64, device=DEV)
        try:
            idx = torch.empty(max(1, 8 * c.n), dtype=torch.int32, device=DEV)
            tot = ctx.neighbours(offs, idx)
        except p3t.P3TError as e:
            if e.code != p3t.P3T_ERR_CAPACITY:
                raise
            idx = torch.empty(max(1, e.total), dtype=torch.int32, device=DEV)
            tot = ctx.neighbours(offs, idx)
        out["offs"] = offs.cpu().numpy()
        out["idx"] = idx[:tot].cpu().numpy()
    if kick_dt is not None:
        vx, vy, vz = to_dev(c.vx), to_dev(c.vy), to_dev(c.vz)
        ctx.kick(kick_dt, *a, vx, vy, vz)
        out["v"] = torch.stack([vx, vy, vz], 1).cpu().numpy()
    ctx.check()
    ctx.close()
    return out


def rel_err(a, ref):
    na = np.linalg.norm(ref, axis=1)
    ok = na > 0
    return np.linalg.norm(a - ref, axis=1)[ok] / na[ok]


def assert_tree_equal(gpu_tree, ref, fp64_moments=True):
    for k in ("keys", "perm", "level", "first", "count", "child", "nchild", "g_first", "g_count"):
        g = gpu_tree[k]
        r = ref[k]
        assert g.shape == r.shape, (k, g.shape, r.shape)
        assert np.array_equal(g, r), k
    for k in ("M", "com", "lo", "hi", "ropen2"):
        assert np.array_equal(gpu_tree[k], ref[k]), k
    if fp64_moments:
        assert np.array_equal(gpu_tree["Q"], ref["Q"]), "Q"
    else:
        # FP32 quadrupole from double-single offsets: relative 2e-5 of the node's
        # quadrupole scale, plus the position resolution of the split
        # (|x - O| ~ R carried to ~2^-46 R), i.e. 1e-12 M R^2 -- a quadrupole error
        # that size moves the force at r >= r_out by < 1e-7 of the monopole term
        qs = np.abs(ref["Q"]).max(axis=1)
        lo = ref["lo"].min(axis=0)
        hi = ref["hi"].max(axis=0)
        R = 0.5 * (hi - lo).max() + 1e-300
        floor = 1e-12 * ref["M"] * R * R
        assert (np.abs(gpu_tree["Q"] - ref["Q"]).max(axis=1) <= 2e-5 * qs + floor + 1e-300).all()


def row_mass_over_r2(x, y, z, m, offs, idx, r_out):
    """Per particle: sum of m_j / r^2 over its row entries with 0 < r < r_out.  The
    scale of an error in K of fixed absolute size (FP32 rounding of K), used as a
    floor when comparing K-weighted sums."""
    n = len(x)
    i = np.repeat(np.arange(n), np.diff(offs))
    j = np.asarray(idx)
    r2 = (x[j] - x[i]) ** 2 + (y[j] - y[i]) ** 2 + (z[j] - z[i]) ** 2
    w = np.where((r2 > 0) & (r2 < r_out ** 2), m[j] / np.where(r2 > 0, r2, 1), 0.0)
    return np.bincount(i, weights=w, minlength=n)
