"""Segregated King W0 = 7 cluster with Kroupa masses (the theta-sweep workload at a
reduced size): both precision forms against the oracle tree, and the tree's
error against the FP64 direct sum falling with theta."""
import numpy as np
import pytest

import oracle
import paper_2110_11658_b300 as p3t
import synth
from gpu_helpers import rel_err, run_gpu

pytestmark = pytest.mark.gpu


def test_king_theta_sweep_precision_forms():
    n = 2 ** 17
    c = synth.make("king", n, 20211022, masses="kroupa", w0=7.0, segregated=True)
    r_out = synth.paper_run_params(n)["r_cut"]
    r_in = 0.1 * r_out
    tg = np.random.default_rng(5).choice(n, 1024, replace=False)
    direct = oracle.direct_split(c.x, c.y, c.z, c.m, r_in, r_out, targets=tg)["far"]
    med_prev = np.inf
    for theta in (0.7, 0.5, 0.3):
        t = oracle.Tree(c.x, c.y, c.z, c.m, theta, r_out, leaf_cap=16, group_size=32)
        f = t.far(r_in)
        for precision in (p3t.P3T_FP32_MIXED, p3t.P3T_FP64):
            prm = p3t.Params(theta=theta, r_in=r_in, r_out=r_out, r_list=r_out, group_size=32,
                             precision=precision)
            g = run_gpu(c, prm, pot=False, nbr=(precision == p3t.P3T_FP32_MIXED and theta == 0.5))
            assert np.array_equal(g["g_cells"], f["n_cell"]) and np.array_equal(g["g_parts"], f["n_part"])
            e = rel_err(g["a"], f["a"])
            if precision == p3t.P3T_FP64:
                assert e.max() < 1e-10
            else:
                assert np.median(e) <= 1e-5 and np.percentile(e, 99) <= 1e-4
            if "offs" in g:
                counts, offs, idx = t.neighbours(r_out)
                assert np.array_equal(g["offs"], offs) and np.array_equal(g["idx"], idx)
        ed = rel_err(f["a"][tg], direct)
        assert np.median(ed) < med_prev
        med_prev = np.median(ed)
    assert med_prev < 1e-4  # theta = 0.3


def test_king_2m_mixed_beats_fp64_at_1e4_p99():
    # the theta-sweep workload at its stated size (King W0 = 7, N = 2^21, Kroupa masses,
    # segregated, r_out = the paper's r_cut) at theta = 0.3: both GPU forms take the same
    # interaction lists, the mixed form agrees with the all-FP64 form within the
    # mixed-precision tolerance, both stay within 1e-4 of the FP64 direct sum at the
    # 99th percentile (1024 seeded targets), and the mixed form is the faster one
    import torch

    from gpu_helpers import DEV, to_dev
    n = 2 ** 21
    c = synth.make("king", n, 20211022, masses="kroupa", w0=7.0, segregated=True)
    r_out = synth.paper_run_params(n)["r_cut"]
    r_in = 0.1 * r_out
    tg = np.random.default_rng(20211022).choice(n, 1024, replace=False)
    direct = oracle.direct_split(c.x, c.y, c.z, c.m, r_in, r_out, targets=tg)["far"]
    d = [to_dev(getattr(c, k)) for k in "xyzm"]
    res = {}
    for name, precision in (("mixed", p3t.P3T_FP32_MIXED), ("fp64", p3t.P3T_FP64)):
        ctx = p3t.Context(p3t.Params(theta=0.3, r_in=r_in, r_out=r_out, r_list=r_out, group_size=32,
                                     precision=precision))
        ctx.set_debug(True)
        ctx.build_tree(*d)
        a = [torch.empty(n, dtype=ctx.acc_dtype, device=DEV) for _ in range(3)]
        ctx.far_force(*a)  # (also counts the neighbours in the mixed form; the timed one only forces)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.far_force(*a)
        e1.record()
        e1.synchronize()
        gc, gp = ctx.group_counts()
        ctx.check()
        res[name] = {"a": torch.stack(a, 1).double().cpu().numpy(), "ms": e0.elapsed_time(e1),
                     "gc": gc.cpu().numpy(), "gp": gp.cpu().numpy()}
        ctx.close()
    m, f = res["mixed"], res["fp64"]
    assert np.array_equal(m["gc"], f["gc"]) and np.array_equal(m["gp"], f["gp"])
    e = rel_err(m["a"], f["a"])
    assert np.median(e) <= 1e-5 and np.percentile(e, 99) <= 1e-4, (np.median(e), np.percentile(e, 99))
    for r in (m, f):
        ed = rel_err(r["a"][tg], direct)
        assert np.percentile(ed, 99) <= 1e-4, np.percentile(ed, 99)
    assert 10 * m["ms"] < f["ms"], (m["ms"], f["ms"])
