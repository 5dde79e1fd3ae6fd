"""B300 (sm_103a) library for the distant-force path of the P3T scheme.

arXiv:2110.11658, Sec. 2: the regular (far) force F_R of Eq. 3 -- Newtonian
gravity weighted by the changeover W = 1 - K of Eq. 6 -- from a Barnes-Hut
tree with opening angle theta (Sec. 2.4), the constant-radius neighbour lists
of Sec. 2.3, and the leapfrog kick of Eq. 12.

Everything runs in hand-written CUDA kernels behind the C ABI of
``include/p3t.h`` (``libp3t.so``).  This package only marshals arguments:
the low-level functions carry the ABI's names (``p3t_create``,
``p3t_build_tree``, ...) and take raw pointers; ``Context`` wraps them for
PyTorch CUDA tensors.  There is no CPU fallback: importing fails if the
shared library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libp3t.so")

P3T_OK = 0
P3T_ERR_INVALID_ARG = 1
P3T_ERR_INVALID_INPUT = 2
P3T_ERR_OOM = 3
P3T_ERR_CAPACITY = 4
P3T_ERR_ORDER = 5
P3T_ERR_TIMEOUT = 6
P3T_ERR_CUDA = 7
P3T_ERR_INTERNAL = 8
P3T_FP32_MIXED = 0
P3T_FP64 = 1

EXPORTED = [
    "p3t_default_params", "p3t_create", "p3t_destroy", "p3t_set_params", "p3t_build_tree",
    "p3t_build_tree_batch",
    "p3t_far_force", "p3t_neighbours", "p3t_neighbours_async", "p3t_kick", "p3t_drift",
    "p3t_step_host", "p3t_status", "p3t_tree_info", "p3t_export_tree", "p3t_group_counts",
    "p3t_set_debug", "p3t_error_string", "p3t_morton_order_noalloc",
    "p3t_graph_capture", "p3t_graph_launch", "p3t_graph_destroy", "p3t_reserve", "p3t_scratch_bytes",
    "p3t_batch_move", "p3t_batch_scatter_neighbours", "p3t_filter_fallbacks", "p3t_irregular",
    "p3t_sample_knn6", "p3t_sample_knn6_brute", "p3t_core_quantities", "p3t_row_mode",
    "p3t_set_spin_limit", "p3t_debug_stalled_scan",
    "p3t_local_bbox", "p3t_key_range_counts", "p3t_partition", "p3t_build_tree_range", "p3t_let_export",
    "p3t_tree_join", "p3t_subtree_boxes",
]
P3T_LET_NODE_BYTES = 288
P3T_LET_PART_BYTES = 96
P3T_NOALLOC_MAX_N = 65536


class p3t_params(C.Structure):
    _fields_ = [("theta", C.c_double), ("r_in", C.c_double), ("r_out", C.c_double),
                ("r_list", C.c_double), ("leaf_cap", C.c_int32), ("group_size", C.c_int32),
                ("tile", C.c_int32), ("threads_per_group", C.c_int32), ("precision", C.c_int32),
                ("quadrupole", C.c_int32)]


class p3t_step_args(C.Structure):
    _fields_ = [("n_clusters", C.c_int32), ("n", C.c_int64), ("seg_offsets", C.c_void_p),
                ("cluster_params", C.c_void_p), ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("m", C.c_void_p), ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p),
                ("ax", C.c_void_p), ("ay", C.c_void_p), ("az", C.c_void_p), ("pot", C.c_void_p),
                ("n_cell", C.c_void_p), ("n_part", C.c_void_p), ("offsets", C.c_void_p), ("idx", C.c_void_p),
                ("capacity", C.c_int64), ("total", C.c_void_p), ("kick_dt", C.c_double),
                ("drift_dt", C.c_double), ("events", C.c_void_p * 5), ("lists_first", C.c_int32)]


class p3t_seg_array(C.Structure):
    _fields_ = [("arena", C.c_void_p), ("batch", C.c_void_p), ("elem_bytes", C.c_int32)]


class P3TError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s failed: %s (code %d)" % (where, p3t_error_string(code), code))


if not os.path.exists(LIB_PATH):
    raise ImportError("libp3t.so is not built (run paper_2110_11658_b300/build.py); "
                      "there is no CPU fallback")
_lib = C.CDLL(LIB_PATH)

_vp = C.c_void_p
_i64 = C.c_int64
_sig = {
    "p3t_default_params": [C.POINTER(p3t_params)],
    "p3t_create": [C.POINTER(_vp), C.POINTER(p3t_params), _vp],
    "p3t_destroy": [_vp],
    "p3t_set_params": [_vp, C.POINTER(p3t_params)],
    "p3t_build_tree": [_vp, _i64, _vp, _vp, _vp, _vp],
    "p3t_build_tree_batch": [_vp, C.c_int32, _i64, _vp, _vp, _vp, _vp, _vp, _vp],
    "p3t_far_force": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "p3t_neighbours": [_vp, _vp, _vp, _i64, C.POINTER(_i64)],
    "p3t_neighbours_async": [_vp, _vp, _vp, _i64, _vp],
    "p3t_kick": [_vp, C.c_double, _vp, _vp, _vp, _vp, _vp, _vp],
    "p3t_drift": [_vp, _i64, C.c_double, _vp, _vp, _vp, _vp, _vp, _vp],
    "p3t_step_host": [_vp, _i64, C.c_double, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                      _vp, _vp, _i64, C.POINTER(_i64)],
    "p3t_status": [_vp],
    "p3t_tree_info": [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64), C.POINTER(C.c_int32)],
    "p3t_export_tree": [_vp] + [_vp] * 15,
    "p3t_group_counts": [_vp, _vp, _vp],
    "p3t_set_debug": [_vp, C.c_int],
    "p3t_set_spin_limit": [_vp, _i64],
    "p3t_debug_stalled_scan": [_vp, _i64],
    "p3t_error_string": [C.c_int],
    "p3t_morton_order_noalloc": [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "p3t_graph_capture": [_vp, C.POINTER(p3t_step_args), C.POINTER(_vp)],
    "p3t_graph_launch": [_vp],
    "p3t_graph_destroy": [_vp],
    "p3t_reserve": [_vp, _i64, C.c_int32],
    "p3t_filter_fallbacks": [_vp, C.POINTER(_i64)],
    "p3t_row_mode": [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "p3t_irregular": [_vp, _i64] + [_vp] * 15,
    "p3t_sample_knn6": [_vp, _i64, _i64, _vp, _vp, _vp],
    "p3t_sample_knn6_brute": [_vp, _i64, _i64, _vp, _vp, _vp],
    "p3t_core_quantities": [_vp, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp],
    "p3t_scratch_bytes": [C.POINTER(p3t_params), _i64, C.c_int32, C.POINTER(_i64)],
    "p3t_batch_move": [_vp, C.c_int32, _i64, _vp, _vp, C.c_int32, C.POINTER(p3t_seg_array), C.c_int32],
    "p3t_batch_scatter_neighbours": [_vp, C.c_int32, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "p3t_local_bbox": [_vp, _i64, _vp, _vp, _vp, C.POINTER(C.c_double)],
    "p3t_key_range_counts": [_vp, _i64, _vp, _vp, _vp, C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_uint64),
                             C.POINTER(C.c_uint64), C.POINTER(_i64)],
    "p3t_partition": [_vp, _i64, _vp, _vp, _vp, C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_uint64),
                      C.c_int32, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_i64)],
    "p3t_build_tree_range": [_vp, _i64, _vp, _vp, _vp, _vp, _vp, C.POINTER(C.c_double), C.c_int32,
                             C.POINTER(C.c_uint64), C.POINTER(C.c_int32)],
    "p3t_subtree_boxes": [_vp, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int32)],
    "p3t_let_export": [_vp, C.c_int32, C.POINTER(C.c_double), C.c_double, _i64, _vp, _i64, _vp, C.POINTER(_i64),
                       C.POINTER(_i64), C.POINTER(C.c_int32)],
    "p3t_tree_join": [_vp, C.c_int32, C.POINTER(_vp), C.POINTER(_i64), C.POINTER(C.c_int32), C.POINTER(_vp),
                      C.POINTER(_i64)],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_char_p if _name == "p3t_error_string" else C.c_int
    globals()[_name] = _f


def p3t_error_string(code: int) -> str:  # noqa: F811  (str instead of bytes)
    return _lib.p3t_error_string(int(code)).decode()


def _check(code: int, where: str):
    if code != P3T_OK:
        raise P3TError(code, where)


@dataclass
class Params:
    """Python view of p3t_params (defaults of p3t_default_params)."""

    theta: float = 0.5
    r_in: float = 0.005
    r_out: float = 0.05
    r_list: float = 0.05
    leaf_cap: int = 16
    group_size: int = 32
    tile: int = 64
    threads_per_group: int = 32
    precision: int = P3T_FP32_MIXED
    quadrupole: int = 1

    def to_c(self) -> p3t_params:
        return p3t_params(self.theta, self.r_in, self.r_out, self.r_list, self.leaf_cap,
                          self.group_size, self.tile, self.threads_per_group, self.precision,
                          self.quadrupole)


def scratch_bytes(params: "Params", n: int, n_clusters: int = 1) -> int:
    """Device bytes a context with these parameters allocates for n particles (p3t_scratch_bytes)."""
    cp = params.to_c()
    b = C.c_int64(0)
    _check(_lib.p3t_scratch_bytes(C.byref(cp), int(n), int(n_clusters), C.byref(b)), "p3t_scratch_bytes")
    return b.value


def batch_move(stream, n_seg, n_batch, batch_off, arena_off, pairs, to_batch):
    """p3t_batch_move: pairs = [(arena_tensor, batch_tensor), ...] (float64 or float32 CUDA tensors)."""
    arr = (p3t_seg_array * len(pairs))()
    for q, (a, b) in enumerate(pairs):
        if a.dtype != b.dtype or a.element_size() not in (4, 8):
            raise ValueError("arena and batch arrays must share a 4- or 8-byte dtype")
        arr[q] = p3t_seg_array(_ptr(a, name="arena"), _ptr(b, name="batch"), a.element_size())
    _check(_lib.p3t_batch_move(C.c_void_p(stream.cuda_stream), int(n_seg), int(n_batch), _ptr(batch_off),
                               _ptr(arena_off), len(pairs), arr, int(bool(to_batch))), "p3t_batch_move")


def batch_scatter_neighbours(stream, n_seg, n_batch, max_entries, batch_off, row_arena_off, ent_arena_off,
                             ent_arena_cap, offsets, idx, arena_offsets, arena_idx, status):
    """p3t_batch_scatter_neighbours on CUDA tensors (see include/p3t.h)."""
    _check(_lib.p3t_batch_scatter_neighbours(
        C.c_void_p(stream.cuda_stream), int(n_seg), int(n_batch), int(max_entries), _ptr(batch_off),
        _ptr(row_arena_off), _ptr(ent_arena_off), _ptr(ent_arena_cap), _ptr(offsets), _ptr(idx),
        _ptr(arena_offsets), _ptr(arena_idx), _ptr(status)), "p3t_batch_scatter_neighbours")


def _ptr(t, dtype=None, n=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (checked), or None."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if n is not None and t.numel() < n:
        raise ValueError("%s has %d elements, needs %d" % (name, t.numel(), n))
    return t.data_ptr()


class Context:
    """One p3t_ctx bound to a CUDA stream (torch's current stream by default)."""

    def __init__(self, params: Params | None = None, stream=None):
        import torch
        self._torch = torch
        self.params = params or Params()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        cp = self.params.to_c()
        _check(_lib.p3t_create(C.byref(h), C.byref(cp), C.c_void_p(stream.cuda_stream)), "p3t_create")
        self._h = h
        self.n = 0
        self._graphs = []

    def close(self):
        for g in getattr(self, "_graphs", []):
            g.close()
        self._graphs = []
        if getattr(self, "_h", None):
            _lib.p3t_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def acc_dtype(self):
        t = self._torch
        return t.float64 if self.params.precision == P3T_FP64 else t.float32

    def set_params(self, params: Params):
        cp = params.to_c()
        _check(_lib.p3t_set_params(self._h, C.byref(cp)), "p3t_set_params")
        self.params = params

    def reserve(self, n: int, n_clusters: int = 1):
        """Size the scratch for n particles in n_clusters clusters now (p3t_reserve)."""
        _check(_lib.p3t_reserve(self._h, int(n), int(n_clusters)), "p3t_reserve")

    # ---- one cluster over several ranks (include/p3t.h; orchestration in decomp.py)
    def local_bbox(self, x, y, z):
        """Exact min xyz, max xyz of the n device points (p3t_local_bbox)."""
        n = x.numel()
        box = (C.c_double * 6)()
        _check(_lib.p3t_local_bbox(self._h, n, _ptr(x, self._torch.float64, n, "x"), _ptr(y, self._torch.float64, n, "y"),
                                   _ptr(z, self._torch.float64, n, "z"), box), "p3t_local_bbox")
        return list(box)

    def key_range_counts(self, x, y, z, global_box, lo, hi):
        """Points per key interval [lo[r], hi[r]) in the cube of global_box (p3t_key_range_counts)."""
        n = 0 if x is None else x.numel()
        nr = len(lo)
        clo, chi = (C.c_uint64 * nr)(*lo), (C.c_uint64 * nr)(*hi)
        out = (C.c_int64 * nr)()
        gb = (C.c_double * 6)(*global_box)
        _check(_lib.p3t_key_range_counts(self._h, n, _ptr(x), _ptr(y), _ptr(z), gb, nr, clo, chi, out),
               "p3t_key_range_counts")
        return list(out)

    def partition(self, x, y, z, global_box, bounds, arrays):
        """The particles packed by destination rank (p3t_partition): arrays is a list of
        8-byte-element CUDA tensors of n elements; returns (packed tensors, counts)."""
        t = self._torch
        n = x.numel()
        nb = len(bounds) - 1
        cb = (C.c_uint64 * (nb + 1))(*bounds)
        dst = [t.empty_like(a) for a in arrays]
        for a in arrays:
            if a.element_size() != 8 or a.numel() != n:
                raise ValueError("partition arrays must hold n 8-byte elements")
        src_p = (_vp * len(arrays))(*[_ptr(a) for a in arrays])
        dst_p = (_vp * len(arrays))(*[_ptr(a) for a in dst])
        cnt = (C.c_int64 * nb)()
        gb = (C.c_double * 6)(*global_box)
        _check(_lib.p3t_partition(self._h, n, _ptr(x), _ptr(y), _ptr(z), gb, nb, cb, len(arrays), src_p, dst_p, cnt),
               "p3t_partition")
        return dst, list(cnt)

    def build_tree_range(self, x, y, z, m, gid, global_box, top_keys, top_levels):
        """This rank's tree of a decomposed cluster (p3t_build_tree_range)."""
        t = self._torch
        n = x.numel()
        nt = len(top_keys)
        tk = (C.c_uint64 * max(1, nt))(*top_keys)
        tl = (C.c_int32 * max(1, nt))(*top_levels)
        gb = (C.c_double * 6)(*global_box)
        _check(_lib.p3t_build_tree_range(self._h, n, _ptr(x, t.float64, n, "x"), _ptr(y, t.float64, n, "y"),
                                         _ptr(z, t.float64, n, "z"), _ptr(m, t.float64, n, "m"),
                                         _ptr(gid, t.int64, n, "gid"), gb, nt, tk, tl), "p3t_build_tree_range")
        self.n = n

    def subtree_boxes(self):
        """Boxes of this rank's subtree roots (p3t_subtree_boxes): a list of 6-tuples."""
        n = C.c_int32(0)
        code = _lib.p3t_subtree_boxes(self._h, 0, None, C.byref(n))
        if code not in (P3T_OK, P3T_ERR_CAPACITY):
            _check(code, "p3t_subtree_boxes")
        buf = (C.c_double * max(6, 6 * n.value))()
        _check(_lib.p3t_subtree_boxes(self._h, n.value, buf, C.byref(n)), "p3t_subtree_boxes")
        return [tuple(buf[6 * i:6 * i + 6]) for i in range(n.value)]

    def let_export(self, boxes, r_halo):
        """The locally essential tree of this rank for a receiver with subtree boxes `boxes`
        (p3t_let_export): (node bytes, particle bytes, n_nodes, n_roots, n_parts)."""
        t = self._torch
        nb = len(boxes)
        cb = (C.c_double * (6 * nb))(*[v for b in boxes for v in b])
        nn, npt, nr = C.c_int64(0), C.c_int64(0), C.c_int32(0)
        code = _lib.p3t_let_export(self._h, nb, cb, float(r_halo), 0, None, 0, None, C.byref(nn), C.byref(npt),
                                   C.byref(nr))
        if code not in (P3T_OK, P3T_ERR_CAPACITY):
            _check(code, "p3t_let_export")
        nodes = t.empty(max(1, nn.value) * P3T_LET_NODE_BYTES, dtype=t.uint8, device="cuda")
        parts = t.empty(max(1, npt.value) * P3T_LET_PART_BYTES, dtype=t.uint8, device="cuda")
        n2, p2 = C.c_int64(0), C.c_int64(0)
        _check(_lib.p3t_let_export(self._h, nb, cb, float(r_halo), max(1, nn.value), _ptr(nodes), max(1, npt.value),
                                   _ptr(parts), C.byref(n2), C.byref(p2), C.byref(nr)), "p3t_let_export")
        return nodes, parts, n2.value, nr.value, p2.value

    def tree_join(self, lets):
        """Join the locally essential trees of the other ranks (p3t_tree_join); lets is a
        list of (node bytes, particle bytes, n_nodes, n_roots, n_parts)."""
        k = len(lets)
        nodes = (_vp * max(1, k))(*[_ptr(a[0]) for a in lets])
        parts = (_vp * max(1, k))(*[_ptr(a[1]) for a in lets])
        nn = (C.c_int64 * max(1, k))(*[int(a[2]) for a in lets])
        nr = (C.c_int32 * max(1, k))(*[int(a[3]) for a in lets])
        npt = (C.c_int64 * max(1, k))(*[int(a[4]) for a in lets])
        _check(_lib.p3t_tree_join(self._h, k, nodes, nn, nr, parts, npt), "p3t_tree_join")

    def set_spin_limit(self, polls: int):
        _check(_lib.p3t_set_spin_limit(self._h, int(polls)), "p3t_set_spin_limit")

    def set_debug(self, on: bool):
        _check(_lib.p3t_set_debug(self._h, int(bool(on))), "p3t_set_debug")

    def build_tree(self, x, y, z, m):
        t = self._torch
        n = x.numel()
        args = [_ptr(a, t.float64, n, nm) for a, nm in zip((x, y, z, m), "xyzm")]
        _check(_lib.p3t_build_tree(self._h, n, *args), "p3t_build_tree")
        self.n = n

    def build_tree_batch(self, seg_offsets, x, y, z, m, cluster_params=None):
        """Ensemble build: seg_offsets is a CUDA int64 tensor of n_clusters + 1 offsets;
        cluster_params an optional CUDA float64 (n_clusters, 4) tensor {theta, r_in, r_out, r_list}."""
        t = self._torch
        n = x.numel()
        nc = seg_offsets.numel() - 1
        args = [_ptr(a, t.float64, n, nm) for a, nm in zip((x, y, z, m), "xyzm")]
        cp = _ptr(cluster_params, t.float64, 4 * nc, "cluster_params")
        _check(_lib.p3t_build_tree_batch(self._h, nc, n, _ptr(seg_offsets, t.int64, nc + 1, "seg_offsets"),
                                         cp, *args), "p3t_build_tree_batch")
        self.n = n

    def far_force(self, ax, ay, az, pot=None, n_cell=None, n_part=None):
        t = self._torch
        d = self.acc_dtype
        _check(_lib.p3t_far_force(self._h, _ptr(ax, d, self.n, "ax"), _ptr(ay, d, self.n, "ay"),
                                  _ptr(az, d, self.n, "az"), _ptr(pot, t.float64, self.n, "pot"),
                                  _ptr(n_cell, t.int64, 1, "n_cell"), _ptr(n_part, t.int64, 1, "n_part")),
               "p3t_far_force")

    def neighbours(self, offsets, idx, capacity=None):
        """Synchronous: returns the total number of entries (raises on capacity)."""
        t = self._torch
        cap = idx.numel() if (idx is not None and capacity is None) else int(capacity or 0)
        tot = C.c_int64(0)
        code = _lib.p3t_neighbours(self._h, _ptr(offsets, t.int64, self.n + 1, "offsets"),
                                   _ptr(idx, t.int32, cap, "idx") if idx is not None else None,
                                   cap, C.byref(tot))
        if code == P3T_ERR_CAPACITY:
            err = P3TError(code, "p3t_neighbours")
            err.total = tot.value
            raise err
        _check(code, "p3t_neighbours")
        return tot.value

    def neighbours_async(self, offsets, idx, total_dev, capacity=None):
        t = self._torch
        cap = idx.numel() if capacity is None else int(capacity)
        _check(_lib.p3t_neighbours_async(self._h, _ptr(offsets, t.int64, self.n + 1, "offsets"),
                                         _ptr(idx, t.int32, cap, "idx"), cap,
                                         _ptr(total_dev, t.int64, 1, "total")),
               "p3t_neighbours_async")

    def kick(self, dt, ax, ay, az, vx, vy, vz):
        t = self._torch
        d = self.acc_dtype
        _check(_lib.p3t_kick(self._h, float(dt), _ptr(ax, d, self.n, "ax"), _ptr(ay, d, self.n, "ay"),
                             _ptr(az, d, self.n, "az"), _ptr(vx, t.float64, self.n, "vx"),
                             _ptr(vy, t.float64, self.n, "vy"), _ptr(vz, t.float64, self.n, "vz")),
               "p3t_kick")

    def drift(self, dt, x, y, z, vx, vy, vz):
        t = self._torch
        n = x.numel()
        _check(_lib.p3t_drift(self._h, n, float(dt), *[_ptr(a, t.float64, n) for a in (x, y, z, vx, vy, vz)]),
               "p3t_drift")

    def step_host(self, dt, x, y, z, m, vx, vy, vz, ax, ay, az, offsets, idx):
        """p3t_step_host on (preferably pinned) CPU tensors; returns the neighbour total."""
        n = x.numel()
        for a in (x, y, z, m, vx, vy, vz, ax, ay, az, offsets, idx):
            if a.is_cuda or not a.is_contiguous():
                raise ValueError("step_host takes contiguous host tensors")
        tot = C.c_int64(0)
        code = _lib.p3t_step_host(self._h, n, float(dt), *[a.data_ptr() for a in (x, y, z, m, vx, vy, vz, ax, ay, az, offsets, idx)],
                                  idx.numel(), C.byref(tot))
        if code == P3T_ERR_CAPACITY:
            err = P3TError(code, "p3t_step_host")
            err.total = tot.value
            raise err
        _check(code, "p3t_step_host")
        self.n = n
        return tot.value

    def status(self):
        return _lib.p3t_status(self._h)

    def check(self):
        _check(self.status(), "p3t_status")

    def tree_info(self):
        n, nn, ng, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int32()
        _check(_lib.p3t_tree_info(self._h, C.byref(n), C.byref(nn), C.byref(ng), C.byref(d)),
               "p3t_tree_info")
        return {"n": n.value, "n_nodes": nn.value, "n_groups": ng.value, "depth": d.value}

    def export_tree(self):
        """Copy of the built tree as CUDA tensors (same layout as the ABI)."""
        t = self._torch
        info = self.tree_info()
        n, nn, ng = info["n"], info["n_nodes"], info["n_groups"]
        dev = t.device("cuda", t.cuda.current_device())
        o = {
            "keys": t.empty(n, dtype=t.int64, device=dev), "perm": t.empty(n, dtype=t.int32, device=dev),
            "level": t.empty(nn, dtype=t.int32, device=dev), "first": t.empty(nn, dtype=t.int32, device=dev),
            "count": t.empty(nn, dtype=t.int32, device=dev), "child": t.empty(nn, dtype=t.int32, device=dev),
            "nchild": t.empty(nn, dtype=t.int32, device=dev), "M": t.empty(nn, dtype=t.float64, device=dev),
            "com": t.empty(nn, 3, dtype=t.float64, device=dev), "Q": t.empty(nn, 6, dtype=t.float64, device=dev),
            "lo": t.empty(nn, 3, dtype=t.float64, device=dev), "hi": t.empty(nn, 3, dtype=t.float64, device=dev),
            "ropen2": t.empty(nn, dtype=t.float64, device=dev),
            "g_first": t.empty(ng, dtype=t.int32, device=dev), "g_count": t.empty(ng, dtype=t.int32, device=dev),
        }
        order = ["keys", "perm", "level", "first", "count", "child", "nchild", "M", "com", "Q", "lo", "hi",
                 "ropen2", "g_first", "g_count"]
        _check(_lib.p3t_export_tree(self._h, *[o[k].data_ptr() if o[k].numel() else None for k in order]),
               "p3t_export_tree")
        self.check()
        return o

    def irregular(self, offsets, idx, x, y, z, m, vx, vy, vz, f=None, jerk=None):
        """Irregular force F_I (Eq. 1) and its time derivative (Eq. 2) over neighbour
        rows (p3t_irregular); returns (f, jerk) as (3, n) float64 CUDA tensors."""
        t = self._torch
        n = x.numel()
        if f is None:
            f = t.empty(3, n, dtype=t.float64, device=x.device)
        if jerk is None:
            jerk = t.empty(3, n, dtype=t.float64, device=x.device)
        args = [_ptr(a, t.float64, n, nm) for a, nm in zip((x, y, z, m, vx, vy, vz), ("x", "y", "z", "m", "vx", "vy", "vz"))]
        outs = [_ptr(f[q], t.float64, n, "f") for q in range(3)] + [_ptr(jerk[q], t.float64, n, "jerk") for q in range(3)]
        _check(_lib.p3t_irregular(self._h, n, _ptr(offsets, t.int64, n + 1, "offsets"), _ptr(idx, t.int32, None, "idx"),
                                  *args, *outs), "p3t_irregular")
        return f, jerk

    def sample_knn6(self, sample, n=None, brute=False):
        """6 nearest neighbours of the sampled particles among the particles of the
        last build: (idx (s, 6) int32, d2 (s, 6) float64) CUDA tensors.  The tree
        search (p3t_sample_knn6), or with brute=True the brute-force search
        (p3t_sample_knn6_brute); the lists are the same."""
        t = self._torch
        n = self.n if n is None else n
        s = sample.numel()
        idx = t.empty(s, 6, dtype=t.int32, device=sample.device)
        d2 = t.empty(s, 6, dtype=t.float64, device=sample.device)
        name = "p3t_sample_knn6_brute" if brute else "p3t_sample_knn6"
        _check(getattr(_lib, name)(self._h, n, s, _ptr(sample, t.int32, s, "sample"), idx.data_ptr(),
                                   d2.data_ptr()), name)
        return idx, d2

    def core_quantities(self, x, y, z, m, sample, idx6, d26):
        """Core quantities from the sample's 6 nearest neighbours (p3t_core_quantities):
        (rho (s,) CUDA tensor, dict of centre, r_core, rho_core, n_core)."""
        t = self._torch
        n, s = x.numel(), sample.numel()
        rho = t.empty(s, dtype=t.float64, device=x.device)
        out = t.empty(6, dtype=t.float64, device=x.device)
        _check(_lib.p3t_core_quantities(self._h, n, *[_ptr(a, t.float64, n, nm) for a, nm in zip((x, y, z, m), "xyzm")],
                                        s, _ptr(sample, t.int32, s, "sample"), _ptr(idx6, t.int32, 6 * s, "idx6"),
                                        _ptr(d26, t.float64, 6 * s, "d26"), rho.data_ptr(), out.data_ptr()),
               "p3t_core_quantities")
        self.check()
        o = out.cpu().numpy()
        return rho, {"centre": o[:3].copy(), "r_core": float(o[3]), "rho_core": float(o[4]), "n_core": int(o[5])}

    def filter_fallbacks(self) -> int:
        """FP64 decisions taken by the FP32 filters since the last build (diagnostic)."""
        v = C.c_int64(0)
        _check(_lib.p3t_filter_fallbacks(self._h, C.byref(v)), "p3t_filter_fallbacks")
        return v.value

    def row_mode(self):
        """(row_cap, rows_valid) of the neighbour lists' row mode (host values)."""
        cap, valid = C.c_int32(0), C.c_int32(0)
        _check(_lib.p3t_row_mode(self._h, C.byref(cap), C.byref(valid)), "p3t_row_mode")
        return cap.value, valid.value

    def group_counts(self):
        t = self._torch
        ng = self.tree_info()["n_groups"]
        c = t.empty(ng, dtype=t.int64, device="cuda")
        p = t.empty(ng, dtype=t.int64, device="cuda")
        _check(_lib.p3t_group_counts(self._h, c.data_ptr(), p.data_ptr()), "p3t_group_counts")
        self.check()
        return c, p

    def capture_step(self, x, y, z, m, ax, ay, az, seg_offsets=None, cluster_params=None, vx=None, vy=None,
                     vz=None, kick_dt=0.0, drift_dt=0.0, pot=None, n_cell=None, n_part=None, offsets=None,
                     idx=None, total=None, capacity=None, events=None, lists_first=False):
        """Record one step (build, far force, neighbour lists, kick, drift) into a CUDA graph
        (p3t_graph_capture).  The tensors are baked in: replays reuse them.  events: up to
        five torch.cuda.Event (timing) or None, recorded as graph nodes at the step's start,
        after the build, the far force and the lists (lists_first: the lists, then the far
        force), and at its end.  lists_first: the lists before the far force (faster for
        short rows; same results)."""
        t = self._torch
        n = x.numel()
        nc = 1 if seg_offsets is None else seg_offsets.numel() - 1
        d = self.acc_dtype
        cap = (idx.numel() if idx is not None else 0) if capacity is None else int(capacity)
        a = p3t_step_args(
            nc, n, _ptr(seg_offsets, t.int64, nc + 1, "seg_offsets"),
            _ptr(cluster_params, t.float64, 4 * nc, "cluster_params"),
            *[_ptr(v, t.float64, n, nm) for v, nm in zip((x, y, z, m), "xyzm")],
            *[_ptr(v, t.float64, n, nm) for v, nm in zip((vx, vy, vz), ("vx", "vy", "vz"))],
            *[_ptr(v, d, n, nm) for v, nm in zip((ax, ay, az), ("ax", "ay", "az"))],
            _ptr(pot, t.float64, n, "pot"), _ptr(n_cell, t.int64, 1, "n_cell"),
            _ptr(n_part, t.int64, 1, "n_part"), _ptr(offsets, t.int64, n + 1, "offsets"),
            _ptr(idx, t.int32, cap, "idx"), cap, _ptr(total, t.int64, 1, "total"), float(kick_dt),
            float(drift_dt))
        a.lists_first = 1 if lists_first else 0
        for k, ev in enumerate(list(events or [])[:5]):
            if ev is not None:
                if not ev.cuda_event:  # torch creates the event on its first record
                    ev.record(self.stream)
                a.events[k] = ev.cuda_event
        h = C.c_void_p()
        _check(_lib.p3t_graph_capture(self._h, C.byref(a), C.byref(h)), "p3t_graph_capture")
        g = Graph(self, h, n, (x, y, z, m, ax, ay, az, seg_offsets, cluster_params, vx, vy, vz, pot, n_cell,
                               n_part, offsets, idx, total))
        self._graphs.append(g)
        return g


class Graph:
    """A captured step (p3t_graph_*); keeps its tensors alive while it exists."""

    def __init__(self, ctx: Context, handle, n, keep):
        self.ctx = ctx
        self._h = handle
        self.n = n
        self._keep = keep

    def launch(self):
        _check(_lib.p3t_graph_launch(self._h), "p3t_graph_launch")
        self.ctx.n = self.n

    def close(self):
        if getattr(self, "_h", None):
            _lib.p3t_graph_destroy(self._h)
            self._h = None
            self._keep = None
