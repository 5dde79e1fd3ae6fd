"""One step captured into a CUDA graph (p3t_graph_capture / p3t_graph_launch).

A replayed step runs the same kernels on the same buffers as the eager entry
points, so its results must equal the eager step's bit for bit, step after
step (the drift moves the particles between steps)."""
import numpy as np
import pytest
import torch

import paper_2110_11658_b300 as p3t
import synth
from gpu_helpers import DEV, to_dev

pytestmark = pytest.mark.gpu

DT = 1.0 / 256


def _state(c):
    return {k: to_dev(getattr(c, k)).clone() for k in ("x", "y", "z", "m", "vx", "vy", "vz")}


def _buffers(n, dtype, cap):
    return {"a": [torch.zeros(n, dtype=dtype, device=DEV) for _ in range(3)],
            "offs": torch.zeros(n + 1, dtype=torch.int64, device=DEV),
            "idx": torch.zeros(cap, dtype=torch.int32, device=DEV),
            "tot": torch.zeros(1, dtype=torch.int64, device=DEV),
            "nc": torch.zeros(1, dtype=torch.int64, device=DEV),
            "np": torch.zeros(1, dtype=torch.int64, device=DEV)}


def _eager_step(ctx, s, b, seg=None, cprm=None):
    if seg is None:
        ctx.build_tree(s["x"], s["y"], s["z"], s["m"])
    else:
        ctx.build_tree_batch(seg, s["x"], s["y"], s["z"], s["m"], cluster_params=cprm)
    ctx.far_force(*b["a"], n_cell=b["nc"], n_part=b["np"])
    ctx.neighbours_async(b["offs"], b["idx"], b["tot"])
    ctx.kick(DT, *b["a"], s["vx"], s["vy"], s["vz"])
    ctx.drift(DT, s["x"], s["y"], s["z"], s["vx"], s["vy"], s["vz"])


def _snapshot(s, b):
    tot = int(b["tot"].item())
    out = {k: v.cpu().numpy().copy() for k, v in s.items()}
    out.update({"a%d" % i: b["a"][i].cpu().numpy().copy() for i in range(3)})
    out.update({"offs": b["offs"].cpu().numpy().copy(), "idx": b["idx"][:tot].cpu().numpy().copy(),
                "nc": int(b["nc"].item()), "np": int(b["np"].item())})
    return out


def _compare(e, g, exact=True):
    for k in e:
        if exact or k in ("m", "offs", "idx", "nc", "np"):
            assert np.array_equal(np.asarray(e[k]), np.asarray(g[k])), k
        else:  # the same sums split differently between the packed pair lanes
            # accelerations to the mixed form's rounding; velocities and positions by the
            # kick of that difference (dt / 2 times it)
            rt, at = (1e-5, 0.0) if k.startswith("a") else (1e-7, 1e-8)
            assert np.allclose(np.asarray(e[k]), np.asarray(g[k]), rtol=rt, atol=at), k


def _run(prm, clusters, cprm_rows=None, steps=3, lists_first=False, exact=True):
    cat = lambda a: np.concatenate([getattr(c, a) for c in clusters])  # noqa: E731
    c = synth.Cluster(*(cat(a) for a in ("x", "y", "z", "m", "vx", "vy", "vz")))
    seg = None
    cprm = None
    if len(clusters) > 1:
        segn = np.zeros(len(clusters) + 1, np.int64)
        np.cumsum([q.n for q in clusters], out=segn[1:])
        seg = torch.from_numpy(segn).to(DEV)
    if cprm_rows is not None:
        cprm = torch.tensor(cprm_rows, dtype=torch.float64, device=DEV)
    dtype = torch.float64 if prm.precision == p3t.P3T_FP64 else torch.float32
    cap = 400 * c.n
    ctx_e, ctx_g = p3t.Context(prm), p3t.Context(prm)
    se, sg = _state(c), _state(c)
    be, bg = _buffers(c.n, dtype, cap), _buffers(c.n, dtype, cap)
    graph = ctx_g.capture_step(sg["x"], sg["y"], sg["z"], sg["m"], *bg["a"], seg_offsets=seg,
                               cluster_params=cprm, vx=sg["vx"], vy=sg["vy"], vz=sg["vz"], kick_dt=DT,
                               drift_dt=DT, n_cell=bg["nc"], n_part=bg["np"], offsets=bg["offs"],
                               idx=bg["idx"], total=bg["tot"], lists_first=lists_first)
    for _ in range(steps):
        _eager_step(ctx_e, se, be, seg, cprm)
        graph.launch()
        ctx_e.check()
        ctx_g.check()
        _compare(_snapshot(se, be), _snapshot(sg, bg), exact)
    assert ctx_g.tree_info() == ctx_e.tree_info()  # the launch restored the captured tree's state
    ctx_g.close()
    ctx_e.close()


@pytest.mark.parametrize("lists_first", [False, True], ids=["far-first", "lists-first"])
@pytest.mark.parametrize("precision", [p3t.P3T_FP32_MIXED, p3t.P3T_FP64], ids=["mixed", "fp64"])
def test_graph_step_equals_eager_single_cluster(precision, lists_first):
    # the graph with the lists before the far force (their own count pass, a force-only
    # walk) gives the same bits as the eager step in the usual order
    c = synth.plummer(6000, 31, masses="kroupa")
    _run(p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05, precision=precision), [c],
         lists_first=lists_first)


@pytest.mark.parametrize("lists_first", [False, True], ids=["far-first", "lists-first"])
@pytest.mark.parametrize("beyond", [False, True], ids=["r_list=r_out", "one-r_list-beyond"])
def test_graph_step_equals_eager_batch_with_cluster_params(lists_first, beyond):
    # per-cluster parameters, one cluster optionally listing neighbours beyond its
    # r_out: with the lists first (force-only walk) the lists are the same and, for
    # that case, the forces only to rounding (the counting walk stages the cluster's
    # neighbour-only sources with mass 0, which moves the other sources between the
    # packed pair lanes); otherwise every bit is the same
    cl = [synth.make("plummer" if k % 2 == 0 else "king", n, 40 + k, w0=5.0)
          for k, n in enumerate((3000, 700, 5000, 1200))]
    rows = []
    for k, q in enumerate(cl):
        rc = synth.paper_run_params(q.n)["r_cut"]
        rows.append([(0.4, 0.6)[k % 2], 0.1 * rc, rc, rc if (k != 1 or not beyond) else 1.3 * rc])
    exact = not (lists_first and beyond)
    _run(p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05), cl, rows, lists_first=lists_first,
         exact=exact, steps=3 if exact else 1)


def test_graph_refuses_launch_after_scratch_moved():
    small, big = synth.plummer(2000, 5), synth.plummer(20000, 6)
    ctx = p3t.Context(p3t.Params())
    s = _state(small)
    b = _buffers(small.n, torch.float32, 100 * small.n)
    g = ctx.capture_step(s["x"], s["y"], s["z"], s["m"], *b["a"], offsets=b["offs"], idx=b["idx"],
                         total=b["tot"])
    g.launch()
    ctx.check()
    ctx.build_tree(*(to_dev(getattr(big, k)) for k in "xyzm"))  # reallocates the scratch
    with pytest.raises(p3t.P3TError) as e:
        g.launch()
    assert e.value.code == p3t.P3T_ERR_ORDER
    ctx.check()
    ctx.close()


def test_graph_phase_events():
    # events recorded as graph nodes time one launch phase by phase: every phase
    # non-negative, the phases summing to the whole step; the step's results are
    # those of the eager step
    c = synth.plummer(20000, 61)
    prm = p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05)
    se, sg = _state(c), _state(c)
    be, bg = _buffers(c.n, torch.float32, 16 * c.n), _buffers(c.n, torch.float32, 16 * c.n)
    ce, cg = p3t.Context(prm), p3t.Context(prm)
    _eager_step(ce, se, be)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    g = cg.capture_step(sg["x"], sg["y"], sg["z"], sg["m"], *bg["a"], vx=sg["vx"], vy=sg["vy"], vz=sg["vz"],
                        kick_dt=DT, drift_dt=DT, n_cell=bg["nc"], n_part=bg["np"], offsets=bg["offs"],
                        idx=bg["idx"], total=bg["tot"], events=ev)
    g.launch()
    torch.cuda.synchronize()
    ce.check()
    cg.check()
    _compare(_snapshot(se, be), _snapshot(sg, bg))
    phases = [ev[k].elapsed_time(ev[k + 1]) for k in range(4)]
    assert all(p >= 0.0 for p in phases) and phases[1] > 0.0
    assert abs(sum(phases) - ev[0].elapsed_time(ev[4])) < 1e-3
    cg.close()
    ce.close()
