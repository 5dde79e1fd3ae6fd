"""CPU checks of the C ABI: the library loads, exports every declared symbol,
and rejects bad arguments before touching the GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "p3t.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(p3t_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for required in ("p3t_build_tree", "p3t_far_force", "p3t_neighbours", "p3t_kick"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2110_11658_b300 as p3t
    lib = C.CDLL(p3t.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(p3t.EXPORTED) == declared_functions()


def test_error_strings_and_defaults():
    import paper_2110_11658_b300 as p3t
    assert p3t.p3t_error_string(0) == "ok"
    for code in range(1, 9):
        assert p3t.p3t_error_string(code) not in ("ok", "unknown error")
    assert p3t.p3t_error_string(99) == "unknown error"
    prm = p3t.p3t_params()
    assert p3t.p3t_default_params(C.byref(prm)) == 0
    d = p3t.Params()
    assert (prm.theta, prm.r_in, prm.r_out, prm.r_list) == (d.theta, d.r_in, d.r_out, d.r_list)
    assert (prm.leaf_cap, prm.group_size, prm.tile, prm.threads_per_group, prm.precision,
            prm.quadrupole) == (d.leaf_cap, d.group_size, d.tile, d.threads_per_group,
                                d.precision, d.quadrupole)


@pytest.mark.parametrize("field,value", [("theta", -0.1), ("r_in", 0.06), ("r_out", 0.0),
                                         ("leaf_cap", 0), ("group_size", 129), ("tile", 48),
                                         ("threads_per_group", 96), ("threads_per_group", 16),
                                         ("precision", 5),
                                         ("quadrupole", 2), ("r_list", -1.0)])
def test_create_rejects_bad_params_without_gpu(field, value):
    import paper_2110_11658_b300 as p3t
    prm = p3t.Params()
    setattr(prm, field, value)
    cp = prm.to_c()
    h = C.c_void_p()
    assert p3t.p3t_create(C.byref(h), C.byref(cp), None) == p3t.P3T_ERR_INVALID_ARG
    assert not h.value


def test_more_targets_than_threads_is_rejected():
    # beyond one warp a group has one thread per target: G <= threads_per_group
    import paper_2110_11658_b300 as p3t
    cp = p3t.Params(group_size=128, threads_per_group=64).to_c()
    h = C.c_void_p()
    assert p3t.p3t_create(C.byref(h), C.byref(cp), None) == p3t.P3T_ERR_INVALID_ARG
    assert not h.value


def test_null_handles_are_rejected():
    import paper_2110_11658_b300 as p3t
    assert p3t.p3t_build_tree(None, 10, None, None, None, None) == p3t.P3T_ERR_INVALID_ARG
    assert p3t.p3t_far_force(None, None, None, None, None, None, None) == p3t.P3T_ERR_INVALID_ARG
    assert p3t.p3t_kick(None, 0.1, None, None, None, None, None, None) == p3t.P3T_ERR_INVALID_ARG
    assert p3t.p3t_status(None) == p3t.P3T_ERR_INVALID_ARG
    assert p3t.p3t_destroy(None) == p3t.P3T_ERR_INVALID_ARG


def test_library_holds_no_oracle_code():
    # the CUDA library and the oracle share nothing: no orc_ symbol in libp3t
    import subprocess

    import paper_2110_11658_b300 as p3t
    out = subprocess.run(["nm", "-D", p3t.LIB_PATH], capture_output=True, text=True).stdout
    assert "orc_" not in out
    srcdir = os.path.join(ROOT, "paper_2110_11658_b300")
    for dirpath, _, files in os.walk(srcdir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "p3t_oracle" not in text, f
