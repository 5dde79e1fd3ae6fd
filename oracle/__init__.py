"""FP64 CPU oracle of the P3T distant-force path (arXiv:2110.11658, Sec. 2).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2110_11658_b300``) and never imports it.

The arithmetic lives in ``p3t_oracle.c`` (plain C, FP64, no FMA contraction);
this module only marshals numpy arrays through ctypes.  Every function cites
the passage it follows in the C source header:

* ``changeover_W`` / ``changeover_K``  -- Eq. 6 with Eqs. 8-10.
* ``direct_split``                    -- Eqs. 1, 3 (far/near/full, phi).
* ``neighbours_brute``                -- Sec. 2.3 constant neighbour radius.
* ``kick``                            -- Eq. 12.
* ``Tree``                            -- Sec. 2.4 Barnes-Hut tree with opening
  angle theta (rules 1-11 in the C header).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants or brute force (none is unpinned).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build as _build

_LIB = None

_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_I32 = C.POINTER(C.c_int32)
_U64 = C.POINTER(C.c_uint64)


def _lib():
    global _LIB
    if _LIB is None:
        path = _build()
        lib = C.CDLL(path)
        lib.orc_changeover_W.restype = C.c_double
        lib.orc_changeover_W.argtypes = [C.c_double] * 3
        lib.orc_changeover_K.restype = C.c_double
        lib.orc_changeover_K.argtypes = [C.c_double] * 3
        lib.orc_direct_split.argtypes = [C.c_int64, _D, _D, _D, _D, C.c_double, C.c_double,
                                         C.c_int64, _I64, _D, _D, _D, _D]
        lib.orc_neighbours_brute.argtypes = [C.c_int64, _D, _D, _D, C.c_double, C.c_int64, _I64,
                                             _I64, _I64, _I32]
        lib.orc_kick.argtypes = [C.c_int64, C.c_double, _D, _D, _D, _D, _D, _D]
        lib.orc_knn.argtypes = [C.c_int64, _D, _D, _D, C.c_int, C.c_int64, _I32, _I32, _D]
        lib.orc_core_quantities.argtypes = [C.c_int64, _D, _D, _D, _D, C.c_int64, _I32, _I32, _D, _D, _D]
        lib.orc_changeover_dWdx.restype = C.c_double
        lib.orc_changeover_dWdx.argtypes = [C.c_double] * 3
        lib.orc_irregular.argtypes = [C.c_int64, _D, _D, _D, _D, _D, _D, _D, C.c_double, C.c_double,
                                      _I64, _I32, _D, _D, _D, _D]
        lib.orc_bounding_cube.argtypes = [C.c_int64, _D, _D, _D, _D]
        lib.orc_interleave.restype = C.c_uint64
        lib.orc_interleave.argtypes = [C.c_int64] * 3
        lib.orc_morton_keys.argtypes = [C.c_int64, _D, _D, _D, _U64]
        lib.orc_tree_build.restype = C.c_void_p
        lib.orc_tree_build.argtypes = [C.c_int64, _D, _D, _D, _D, C.c_double, C.c_double,
                                       C.c_int, C.c_int]
        lib.orc_tree_free.argtypes = [C.c_void_p]
        lib.orc_tree_n_nodes.restype = C.c_int64
        lib.orc_tree_n_nodes.argtypes = [C.c_void_p]
        lib.orc_tree_n_groups.restype = C.c_int64
        lib.orc_tree_n_groups.argtypes = [C.c_void_p]
        lib.orc_tree_export.argtypes = [C.c_void_p, _U64, _I32, _I32, _I32, _I32, _I32, _I32,
                                        _D, _D, _D, _D, _D, _D, _I32, _I32, _D, _D]
        lib.orc_tree_far.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int64,
                                     _I64, _D, _D, _D, _D, _I64, _I64]
        lib.orc_tree_neighbours.argtypes = [C.c_void_p, C.c_double, C.c_int64, _I64, _I64, _I64,
                                            _I32]
        _LIB = lib
    return _LIB


def _p(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def changeover_W(r: float, r_in: float, r_out: float) -> float:
    """Far weight W = 1 - K of Eq. 6."""
    return _lib().orc_changeover_W(r, r_in, r_out)


def changeover_K(r: float, r_in: float, r_out: float) -> float:
    """Near weight K of Eq. 6."""
    return _lib().orc_changeover_K(r, r_in, r_out)


def direct_split(x, y, z, m, r_in, r_out, targets=None):
    """Direct split sum (Eqs. 1, 3) -> dict(far, near, full (nt,3), pot (nt,))."""
    x, y, z, m = map(_f64, (x, y, z, m))
    n = x.shape[0]
    t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
    nt = t.shape[0]
    far = np.zeros((nt, 3))
    near = np.zeros((nt, 3))
    full = np.zeros((nt, 3))
    pot = np.zeros(nt)
    _lib().orc_direct_split(n, _p(x, _D), _p(y, _D), _p(z, _D), _p(m, _D), r_in, r_out, nt,
                            _p(t, _I64), _p(far, _D), _p(near, _D), _p(full, _D), _p(pot, _D))
    return {"far": far, "near": near, "full": full, "pot": pot}


def neighbours_brute(x, y, z, r_list, targets=None):
    """Neighbour rows (ascending original index) of the targets by brute force."""
    x, y, z = map(_f64, (x, y, z))
    n = x.shape[0]
    t = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
    nt = t.shape[0]
    counts = np.zeros(nt, np.int64)
    lib = _lib()
    lib.orc_neighbours_brute(n, _p(x, _D), _p(y, _D), _p(z, _D), r_list, nt, _p(t, _I64),
                             _p(counts, _I64), None, None)
    offs = np.zeros(nt + 1, np.int64)
    np.cumsum(counts, out=offs[1:])
    idx = np.zeros(max(1, int(offs[-1])), np.int32)
    lib.orc_neighbours_brute(n, _p(x, _D), _p(y, _D), _p(z, _D), r_list, nt, _p(t, _I64),
                             _p(counts, _I64), _p(offs, _I64), _p(idx, _I32))
    return offs, idx[: offs[-1]]


def kick(dt, ax, ay, az, vx, vy, vz):
    """Eq. 12 on copies: returns (vx, vy, vz) + (dt/2) a."""
    vx, vy, vz = (np.array(v, dtype=np.float64, copy=True) for v in (vx, vy, vz))
    ax, ay, az = map(_f64, (ax, ay, az))
    _lib().orc_kick(vx.shape[0], dt, _p(ax, _D), _p(ay, _D), _p(az, _D), _p(vx, _D),
                    _p(vy, _D), _p(vz, _D))
    return vx, vy, vz


def changeover_dWdx(r: float, r_in: float, r_out: float) -> float:
    """dW/dx (the bracket of Eq. 7), 0 outside 0 <= x < 1."""
    return _lib().orc_changeover_dWdx(r, r_in, r_out)


def irregular(x, y, z, m, vx, vy, vz, r_in, r_out, offsets, idx, scales=False):
    """Irregular force F_I (Eq. 1) and jerk dF_I/dt (Eq. 2) over neighbour rows
    (offsets int64[n+1], idx int32).  Returns (f (n,3), jerk (n,3)) and, with
    scales=True, also the per-particle sums of the term magnitudes."""
    x, y, z, m, vx, vy, vz = map(_f64, (x, y, z, m, vx, vy, vz))
    n = x.shape[0]
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if idx.size == 0:
        idx = np.zeros(1, np.int32)
    f = np.zeros((n, 3))
    jerk = np.zeros((n, 3))
    sf = np.zeros(n) if scales else None
    sj = np.zeros(n) if scales else None
    _lib().orc_irregular(n, _p(x, _D), _p(y, _D), _p(z, _D), _p(m, _D), _p(vx, _D), _p(vy, _D),
                         _p(vz, _D), r_in, r_out, _p(offsets, _I64), _p(idx, _I32), _p(f, _D),
                         _p(jerk, _D), _p(sf, _D), _p(sj, _D))
    return (f, jerk, sf, sj) if scales else (f, jerk)


def knn(x, y, z, sample, k=6):
    """k nearest neighbours (FP64 squared distance, ties by index) of the sampled
    particles by brute force: (idx (s, k) int32, d2 (s, k))."""
    x, y, z = map(_f64, (x, y, z))
    sample = np.ascontiguousarray(sample, dtype=np.int32)
    s = sample.shape[0]
    idx = np.zeros((s, k), np.int32)
    d2 = np.zeros((s, k))
    _lib().orc_knn(x.shape[0], _p(x, _D), _p(y, _D), _p(z, _D), k, s, _p(sample, _I32), _p(idx, _I32),
                   _p(d2, _D))
    return idx, d2


def core_quantities(x, y, z, m, sample, idx6, d26):
    """Core quantities from the 6 nearest neighbours of a sample: (rho (s,),
    dict(centre, r_core, rho_core, n_core))."""
    x, y, z, m = map(_f64, (x, y, z, m))
    sample = np.ascontiguousarray(sample, dtype=np.int32)
    idx6 = np.ascontiguousarray(idx6, dtype=np.int32)
    d26 = _f64(d26)
    s = sample.shape[0]
    rho = np.zeros(s)
    out = np.zeros(6)
    _lib().orc_core_quantities(x.shape[0], _p(x, _D), _p(y, _D), _p(z, _D), _p(m, _D), s, _p(sample, _I32),
                               _p(idx6, _I32), _p(d26, _D), _p(rho, _D), _p(out, _D))
    return rho, {"centre": out[:3].copy(), "r_core": out[3], "rho_core": out[4], "n_core": int(out[5])}


def bounding_cube(x, y, z):
    """Rule 1: (min_x, min_y, min_z, side)."""
    x, y, z = map(_f64, (x, y, z))
    out = np.zeros(4)
    _lib().orc_bounding_cube(x.shape[0], _p(x, _D), _p(y, _D), _p(z, _D), _p(out, _D))
    return out


def interleave(qx: int, qy: int, qz: int) -> int:
    """Rule 3 on one triple of 21-bit integers."""
    return int(_lib().orc_interleave(qx, qy, qz))


def morton_keys(x, y, z):
    """Rules 1-3: one 63-bit key per particle (original order)."""
    x, y, z = map(_f64, (x, y, z))
    keys = np.zeros(x.shape[0], np.uint64)
    _lib().orc_morton_keys(x.shape[0], _p(x, _D), _p(y, _D), _p(z, _D), _p(keys, _U64))
    return keys


class Tree:
    """The reference tree (rules 1-8) over FP64 particles."""

    def __init__(self, x, y, z, m, theta, r_out, leaf_cap=16, group_size=64):
        self.x, self.y, self.z, self.m = map(_f64, (x, y, z, m))
        self.n = self.x.shape[0]
        self.theta, self.r_out = float(theta), float(r_out)
        self._h = _lib().orc_tree_build(self.n, _p(self.x, _D), _p(self.y, _D), _p(self.z, _D),
                                        _p(self.m, _D), self.theta, self.r_out, int(leaf_cap),
                                        int(group_size))
        self.n_nodes = int(_lib().orc_tree_n_nodes(self._h))
        self.n_groups = int(_lib().orc_tree_n_groups(self._h))

    def __del__(self):
        if getattr(self, "_h", None):
            _lib().orc_tree_free(self._h)
            self._h = None

    def export(self) -> dict:
        n, nn, ng = self.n, self.n_nodes, self.n_groups
        d = {
            "keys": np.zeros(n, np.uint64), "perm": np.zeros(n, np.int32),
            "level": np.zeros(nn, np.int32), "first": np.zeros(nn, np.int32),
            "count": np.zeros(nn, np.int32), "child": np.zeros(nn, np.int32),
            "nchild": np.zeros(nn, np.int32), "M": np.zeros(nn), "com": np.zeros((nn, 3)),
            "Q": np.zeros((nn, 6)), "lo": np.zeros((nn, 3)), "hi": np.zeros((nn, 3)),
            "ropen2": np.zeros(nn), "g_first": np.zeros(ng, np.int32),
            "g_count": np.zeros(ng, np.int32), "g_lo": np.zeros((ng, 3)),
            "g_hi": np.zeros((ng, 3)),
        }
        _lib().orc_tree_export(
            self._h, _p(d["keys"], _U64), _p(d["perm"], _I32), _p(d["level"], _I32),
            _p(d["first"], _I32), _p(d["count"], _I32), _p(d["child"], _I32),
            _p(d["nchild"], _I32), _p(d["M"], _D), _p(d["com"], _D), _p(d["Q"], _D),
            _p(d["lo"], _D), _p(d["hi"], _D), _p(d["ropen2"], _D), _p(d["g_first"], _I32),
            _p(d["g_count"], _I32), _p(d["g_lo"], _D), _p(d["g_hi"], _D))
        return d

    def far(self, r_in, r_out=None, quadrupole=True, groups=None):
        """Far force on the particles of `groups` (all if None), original order.

        Returns dict(a (n,3) with NaN rows for unselected particles, pot (n,),
        n_cell, n_part (per selected group)).
        """
        r_out = self.r_out if r_out is None else float(r_out)
        g = None if groups is None else np.ascontiguousarray(groups, np.int64)
        ng = self.n_groups if g is None else g.shape[0]
        ax = np.full(self.n, np.nan)
        ay = np.full(self.n, np.nan)
        az = np.full(self.n, np.nan)
        pot = np.full(self.n, np.nan)
        nc = np.zeros(ng, np.int64)
        npart = np.zeros(ng, np.int64)
        _lib().orc_tree_far(self._h, int(bool(quadrupole)), float(r_in), r_out, ng, _p(g, _I64),
                            _p(ax, _D), _p(ay, _D), _p(az, _D), _p(pot, _D), _p(nc, _I64),
                            _p(npart, _I64))
        return {"a": np.stack([ax, ay, az], axis=1), "pot": pot, "n_cell": nc, "n_part": npart}

    def neighbours(self, r_list, groups=None):
        """Neighbour rows by tree search for the particles of `groups`.

        Returns (counts (n,) with -1 for unselected particles, offsets (n+1,),
        idx) where unselected rows are empty.
        """
        g = None if groups is None else np.ascontiguousarray(groups, np.int64)
        ng = self.n_groups if g is None else g.shape[0]
        counts = np.full(self.n, -1, np.int64)
        lib = _lib()
        lib.orc_tree_neighbours(self._h, float(r_list), ng, _p(g, _I64), _p(counts, _I64),
                                None, None)
        c = np.maximum(counts, 0)
        offs = np.zeros(self.n + 1, np.int64)
        np.cumsum(c, out=offs[1:])
        idx = np.zeros(max(1, int(offs[-1])), np.int32)
        counts2 = np.full(self.n, -1, np.int64)
        lib.orc_tree_neighbours(self._h, float(r_list), ng, _p(g, _I64), _p(counts2, _I64),
                                _p(offs, _I64), _p(idx, _I32))
        return counts, offs, idx[: offs[-1]]
