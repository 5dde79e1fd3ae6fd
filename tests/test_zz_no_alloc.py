"""The allocation-free Morton-order entry point against the regular tree build.

p3t_morton_order_noalloc serves callers that cannot allocate device memory
where they need the library (a host whose own pool owns the GPU's memory, or
a loop that must not allocate once running).  Its keys and sort permutation
must equal what p3t_build_tree computes, on consecutive calls that reuse the
library's one static scratch array.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import paper_2110_11658_b300 as p3t
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _regular(c):
    """keys and perm from p3t_build_tree + p3t_export_tree."""
    ctx = p3t.Context(p3t.Params())
    ctx.build_tree(_dev(c.x), _dev(c.y), _dev(c.z), _dev(c.m))
    t = ctx.export_tree()
    out = t["keys"].cpu().numpy().view(np.uint64), t["perm"].cpu().numpy()
    ctx.close()
    return out


def _noalloc(c):
    x, y, z, m = _dev(c.x), _dev(c.y), _dev(c.z), _dev(c.m)
    keys = torch.full((c.n,), -1, dtype=torch.int64, device=DEV)
    perm = torch.full((c.n,), -1, dtype=torch.int32, device=DEV)
    stream = torch.cuda.current_stream(DEV)
    code = p3t.p3t_morton_order_noalloc(c.n, x.data_ptr(), y.data_ptr(), z.data_ptr(), m.data_ptr(),
                                        keys.data_ptr(), perm.data_ptr(), C.c_void_p(stream.cuda_stream))
    return code, keys.cpu().numpy().view(np.uint64), perm.cpu().numpy()


def test_noalloc_equals_build_tree_on_consecutive_calls():
    torch.cuda.set_device(DEV)
    first = synth.plummer(50000, 101, masses="kroupa")
    second = synth.king(7001, 102, 7.0)  # a smaller second call: leftovers must not matter
    for c in (first, second, first):
        code, keys, perm = _noalloc(c)
        assert code == p3t.P3T_OK, p3t.p3t_error_string(code)
        rk, rp = _regular(c)
        assert np.array_equal(keys, rk)
        assert np.array_equal(perm, rp)
        # and directly against the oracle's keys, stably ordered by (key, index)
        ok = oracle.morton_keys(c.x, c.y, c.z)
        order = np.lexsort((np.arange(c.n), ok))
        assert np.array_equal(perm, order) and np.array_equal(keys, ok[order])


def test_noalloc_rejects_sizes_beyond_its_array():
    torch.cuda.set_device(DEV)
    n = p3t.P3T_NOALLOC_MAX_N + 1
    buf = torch.zeros(n, dtype=torch.float64, device=DEV)
    keys = torch.zeros(n, dtype=torch.int64, device=DEV)
    perm = torch.zeros(n, dtype=torch.int32, device=DEV)
    code = p3t.p3t_morton_order_noalloc(n, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                        buf.data_ptr(), keys.data_ptr(), perm.data_ptr(), None)
    assert code == p3t.P3T_ERR_CAPACITY
    # the largest allowed size still works
    c = synth.plummer(p3t.P3T_NOALLOC_MAX_N, 103)
    code, keys2, perm2 = _noalloc(c)
    assert code == p3t.P3T_OK
    rk, rp = _regular(c)
    assert np.array_equal(keys2, rk) and np.array_equal(perm2, rp)


def test_noalloc_invalid_input_does_not_carry_over():
    # a NaN position is reported; the next valid call on the same shared array
    # starts clean and returns the regular build's keys and permutation
    torch.cuda.set_device(DEV)
    bad = synth.plummer(3000, 104)
    bad.x[1234] = np.nan
    code, _, _ = _noalloc(bad)
    assert code == p3t.P3T_ERR_INVALID_INPUT
    good = synth.plummer(3000, 105)
    code, keys, perm = _noalloc(good)
    assert code == p3t.P3T_OK
    rk, rp = _regular(good)
    assert np.array_equal(keys, rk) and np.array_equal(perm, rp)
