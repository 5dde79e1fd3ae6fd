"""Error paths of the C ABI on the GPU: invalid inputs latched on the device,
call order, capacity reporting, and the host-buffer step.  No test faults,
traps or hangs the GPU: every error is a returned status."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import paper_2110_11658_b300 as p3t
import synth
from gpu_helpers import DEV, run_gpu, to_dev

pytestmark = pytest.mark.gpu


def test_far_force_before_build_is_an_order_error():
    ctx = p3t.Context(p3t.Params())
    a = torch.empty(10, dtype=torch.float32, device=DEV)
    with pytest.raises(p3t.P3TError) as e:
        ctx.far_force(a, a, a)
    assert e.value.code == p3t.P3T_ERR_ORDER
    off = torch.empty(11, dtype=torch.int64, device=DEV)
    assert p3t.p3t_neighbours(ctx.handle, off.data_ptr(), None, 0, C.byref(C.c_int64())) == p3t.P3T_ERR_ORDER


@pytest.mark.parametrize("bad", ["nan_x", "inf_z", "neg_mass", "nan_mass"])
def test_invalid_input_is_latched(bad):
    c = synth.plummer(1000, 1)
    if bad == "nan_x":
        c.x[17] = np.nan
    elif bad == "inf_z":
        c.z[999] = np.inf
    elif bad == "neg_mass":
        c.m[3] = -1e-3
    else:
        c.m[0] = np.nan
    ctx = p3t.Context(p3t.Params())
    ctx.build_tree(to_dev(c.x), to_dev(c.y), to_dev(c.z), to_dev(c.m))
    a = [torch.empty(1000, dtype=torch.float32, device=DEV) for _ in range(3)]
    ctx.far_force(*a)  # runs to completion on garbage, never faults
    assert ctx.status() == p3t.P3T_ERR_INVALID_INPUT
    assert ctx.status() == p3t.P3T_OK  # the latch clears once read
    # the context stays usable
    g = synth.plummer(1000, 2)
    ctx.build_tree(to_dev(g.x), to_dev(g.y), to_dev(g.z), to_dev(g.m))
    ctx.far_force(*a)
    ctx.check()


def test_neighbour_capacity_reports_total():
    c = synth.plummer(4096, 5)
    ctx = p3t.Context(p3t.Params(r_list=0.08))
    ctx.build_tree(to_dev(c.x), to_dev(c.y), to_dev(c.z), to_dev(c.m))
    offs = torch.empty(4097, dtype=torch.int64, device=DEV)
    small = torch.full((10,), -7, dtype=torch.int32, device=DEV)
    with pytest.raises(p3t.P3TError) as e:
        ctx.neighbours(offs, small)
    o2, i2 = oracle.neighbours_brute(c.x, c.y, c.z, 0.08)
    assert e.value.code == p3t.P3T_ERR_CAPACITY and e.value.total == o2[-1]
    assert np.array_equal(offs.cpu().numpy(), o2)
    assert (small.cpu().numpy() == -7).all()  # nothing written beyond (or within) capacity
    # asynchronous variant: no entry written, error latched
    tot = torch.zeros(1, dtype=torch.int64, device=DEV)
    ctx.neighbours_async(offs, small, tot)
    assert ctx.status() == p3t.P3T_ERR_CAPACITY
    assert int(tot.item()) == o2[-1] and (small.cpu().numpy() == -7).all()
    big = torch.empty(int(o2[-1]), dtype=torch.int32, device=DEV)
    ctx.neighbours_async(offs, big, tot)
    ctx.check()
    assert np.array_equal(big.cpu().numpy(), i2)


def test_step_host_equals_device_path():
    c = synth.plummer(8192, 21, masses="kroupa")
    prm = p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05)
    dt = 1.0 / 256
    g = run_gpu(c, prm, kick_dt=dt)
    ctx = p3t.Context(prm)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    x, y, z, m = pin(c.x), pin(c.y), pin(c.z), pin(c.m)
    vx, vy, vz = pin(c.vx), pin(c.vy), pin(c.vz)
    a = [torch.empty(c.n, dtype=torch.float32).pin_memory() for _ in range(3)]
    offs = torch.empty(c.n + 1, dtype=torch.int64).pin_memory()
    idx = torch.empty(8 * c.n, dtype=torch.int32).pin_memory()
    tot = ctx.step_host(dt, x, y, z, m, vx, vy, vz, *a, offs, idx)
    assert np.array_equal(torch.stack(a, 1).double().numpy(), g["a"])
    assert np.array_equal(torch.stack([vx, vy, vz], 1).numpy(), g["v"])
    assert np.array_equal(offs.numpy(), g["offs"]) and np.array_equal(idx[:tot].numpy(), g["idx"])


def test_kick_and_drift_exact():
    rng = np.random.default_rng(8)
    n = 5000
    c = synth.plummer(n, 8)
    ctx = p3t.Context(p3t.Params(precision=p3t.P3T_FP64))
    ctx.build_tree(to_dev(c.x), to_dev(c.y), to_dev(c.z), to_dev(c.m))
    a = rng.normal(size=(3, n))
    v = [to_dev(c.vx), to_dev(c.vy), to_dev(c.vz)]
    ctx.kick(1.0 / 512, *[to_dev(q) for q in a], *v)
    ref = oracle.kick(1.0 / 512, *a, c.vx, c.vy, c.vz)
    for got, r in zip(v, ref):
        assert np.array_equal(got.cpu().numpy(), r)
    x = [to_dev(c.x), to_dev(c.y), to_dev(c.z)]
    ctx.drift(0.01, *x, *v)
    ctx.check()
    assert np.array_equal(x[0].cpu().numpy(), c.x + 0.01 * ref[0])


def test_bounded_wait_runs_out_and_returns_a_status():
    # a prefix sum whose first tile is never handed out: the look-back waits of the
    # tiles after it poll a status word that nothing writes, give up after the
    # context's spin limit, latch P3T_ERR_TIMEOUT and finish; the context stays usable
    ctx = p3t.Context(p3t.Params(theta=0.5, r_in=0.005, r_out=0.05, r_list=0.05))
    ctx.reserve(20000)
    assert p3t.p3t_debug_stalled_scan(ctx.handle, 0) == p3t.P3T_ERR_INVALID_ARG
    assert p3t.p3t_debug_stalled_scan(ctx.handle, 10 ** 6) == p3t.P3T_ERR_ORDER  # beyond the scratch
    assert p3t.p3t_set_spin_limit(ctx.handle, -1) == p3t.P3T_ERR_INVALID_ARG
    ctx.set_spin_limit(2000)
    for n in (5000, 20000):  # 3 and 10 tiles of the scan
        assert p3t.p3t_debug_stalled_scan(ctx.handle, n) == p3t.P3T_ERR_TIMEOUT
        assert ctx.status() == p3t.P3T_OK  # read once, cleared
    ctx.set_spin_limit(0)  # the default again
    c = synth.plummer(4096, synth.BASE_SEED)
    g = run_gpu(c, ctx.params, nbr=True)
    ctx.build_tree(to_dev(c.x), to_dev(c.y), to_dev(c.z), to_dev(c.m))
    a = [torch.empty(c.n, dtype=torch.float32, device=DEV) for _ in range(3)]
    ctx.far_force(*a)
    offs = torch.empty(c.n + 1, dtype=torch.int64, device=DEV)
    idx = torch.empty(8 * c.n, dtype=torch.int32, device=DEV)
    tot = ctx.neighbours(offs, idx)
    ctx.check()
    assert np.array_equal(torch.stack(a, 1).double().cpu().numpy(), g["a"])
    assert np.array_equal(offs.cpu().numpy(), g["offs"]) and np.array_equal(idx[:tot].cpu().numpy(), g["idx"])
    ctx.close()
