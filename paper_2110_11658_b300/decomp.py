"""One cluster over several ranks: the multi-GPU distant-force step (the force
calculator's multi-GPU extension that Sec. 4 of the paper names as future work).

Rank r holds the particles whose Morton keys (rules 1-3, on the bounding box of
the whole cluster) lie in [b_r, b_{r+1}).  The splitters are cell boundaries of
the global octree: descending from the root towards the key-order quantile
N r / P, a cell is entered while it holds more than max(16 G, leaf_cap)
particles (so it may straddle the splitter and be split in any build) and the
splitter is put at the nearer edge of the first child that holds fewer.  Every
cell that straddles a splitter ("top cell") therefore holds more than that
threshold: it is split, never cut into walk groups, and the rest of the global
tree is complete subtrees owned by single ranks.  Each rank then

1. builds its part of the tree (top cells forced open, order (key, global index)),
2. sends every other rank the locally essential tree of its subtrees as that
   rank's subtree boxes see them (the opening rule of Sec. 2.4 with r_out, or the
   list radius when larger, so the neighbour halo is included; every group of the
   receiver lies in one of those boxes, so the tree holds whatever any of them opens),
3. joins what it receives: the top cells' moments follow from the joined
   children, and its groups walk the global tree.

Interaction lists, forces and neighbour rows (global indices) equal those of one
build of the whole cluster.  Every step that touches particles or nodes runs in
the library's kernels; this module only decides splitters and top cells from
reduced counts and moves buffers between ranks.

Two ways to run the same code: ``TorchComm`` (one process per GPU,
torch.distributed: NCCL for device buffers, gloo on the CPU) and ``LocalComm``
(all ranks in one process, e.g. on one GPU: collectives become list operations,
"sending" a buffer hands it over on the same device).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

LEVELS = 21
KEY_END = 1 << 63
GROUP_NODE_FACTOR = 16


def cell_bounds(level: int, key: int):
    """[first, end) keys of the level-`level` cell holding `key`."""
    shift = 63 - 3 * level
    first = (key >> shift) << shift
    return first, first + (1 << shift)


# ---------------------------------------------------------------------------- communicators
class LocalComm:
    """All ranks in this process: every call takes and returns one value per rank."""

    def __init__(self, size: int):
        self.size = size
        self.ranks = list(range(size))

    def allreduce(self, values, op):
        a = np.stack([np.asarray(v) for v in values])
        r = {"sum": a.sum(0), "min": a.min(0), "max": a.max(0)}[op]
        return [r.copy() for _ in values]

    def allgather(self, values):
        return [list(values) for _ in values]

    def alltoall(self, send):
        """send[i][d]: what rank i sends to rank d; returns recv[d][i]."""
        return [[send[i][d] for i in range(self.size)] for d in range(self.size)]


class TorchComm:
    """One rank per process over torch.distributed.  Device tensors travel by the
    process group's backend (NCCL); host numbers by all_reduce / all_gather_object."""

    def __init__(self, dist, device=None):
        self.dist = dist
        self.size = dist.get_world_size()
        self.ranks = [dist.get_rank()]
        self.device = device

    def allreduce(self, values, op):
        import torch
        (v,) = values
        a = np.asarray(v)
        dt = torch.int64 if a.dtype.kind in "iu" else torch.float64
        t = torch.tensor(a.reshape(-1), dtype=dt, device=self.device if self.device is not None else "cpu")
        red = {"sum": self.dist.ReduceOp.SUM, "min": self.dist.ReduceOp.MIN, "max": self.dist.ReduceOp.MAX}[op]
        self.dist.all_reduce(t, op=red)
        return [t.cpu().numpy().astype(a.dtype).reshape(a.shape)]

    def allgather(self, values):
        (v,) = values
        out = [None] * self.size
        self.dist.all_gather_object(out, v)
        return [out]

    def alltoall(self, send):
        """send[0][d] (torch tensors, 1-D, any dtype): point-to-point exchange, sizes
        first; returns [[received from rank s for s in ranks]]."""
        import torch
        (row,) = send
        me = self.ranks[0]
        sizes = self.allgather([[int(t.numel()) for t in row]])[0]
        recv = [None] * self.size
        ops = []
        for s in range(self.size):
            if s == me:
                recv[s] = row[s]
                continue
            recv[s] = torch.empty(sizes[s][me], dtype=row[s].dtype, device=row[s].device)
            if recv[s].numel() > 0:
                ops.append(self.dist.P2POp(self.dist.irecv, recv[s], s))
            if row[s].numel() > 0:
                ops.append(self.dist.P2POp(self.dist.isend, row[s].contiguous(), s))
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()
        return [recv]


# ---------------------------------------------------------------------------- splitters
def choose_splitters(n_total: int, n_ranks: int, threshold: int, global_counts):
    """Splitter keys b_1 .. b_{P-1} (plus b_0 = 0 and b_P = 2^63).

    global_counts(ranges) -> particles of the whole cluster per key interval.  All
    splitters descend together from the root, one reduction per level: the child
    holding the target position (N s / P particles before the splitter) is entered
    while it holds more than `threshold` particles and lies above level 21; else the
    splitter takes the nearer edge of that child.  Every cell a splitter ends up
    inside was entered, so it holds more than `threshold` particles."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be positive")
    if n_ranks == 1:
        return [0, KEY_END]
    if n_total <= threshold:
        raise ValueError("%d particles cannot be split: the root holds no more than %d" % (n_total, threshold))
    targets = [(n_total * s) // n_ranks for s in range(1, n_ranks)]
    # per splitter: (level, first key, particles before the cell), or the final key
    cells = [(0, 0, 0) for _ in targets]
    final = [None] * len(targets)
    while any(f is None for f in final):
        active = [i for i, f in enumerate(final) if f is None]
        ranges = []
        for i in active:
            level, first, _ = cells[i]
            size = 1 << (63 - 3 * (level + 1))
            ranges += [(first + o * size, first + (o + 1) * size) for o in range(8)]
        counts = global_counts(ranges)
        for a, i in enumerate(active):
            level, first, before = cells[i]
            q = targets[i]
            cum = before
            for o in range(8):
                c = int(counts[8 * a + o])
                lo, hi = ranges[8 * a + o]
                if q < cum + c or o == 7:
                    if q <= cum:
                        final[i] = lo
                    elif c > threshold and level + 1 < LEVELS:
                        cells[i] = (level + 1, lo, cum)
                    else:
                        final[i] = lo if q - cum <= cum + c - q else hi
                    break
                cum += c
    bounds = [0] + final + [KEY_END]
    for a, b in zip(bounds, bounds[1:]):
        if not a < b:
            raise ValueError("a rank would hold no particle (splitters %s)" % bounds)
    return bounds


def top_cells(bounds, global_counts):
    """The cells that straddle a splitter with particles on both sides: [(key, level)]
    sorted by (level, key).  global_counts as in choose_splitters."""
    cand = []
    for b in bounds[1:-1]:
        for level in range(LEVELS):
            first, end = cell_bounds(level, b)
            if first == b:  # aligned here, so at every deeper level too
                break
            cand.append((level, first, end, b))
    if not cand:
        return []
    ranges = []
    for level, first, end, b in cand:
        ranges += [(first, b), (b, end)]
    counts = global_counts(ranges)
    tops = set()
    for a, (level, first, end, b) in enumerate(cand):
        if counts[2 * a] > 0 and counts[2 * a + 1] > 0:
            tops.add((level, first))
    return [(k, l) for l, k in sorted(tops)]


# ---------------------------------------------------------------------------- the step
@dataclass
class RankPart:
    """One rank's particles (device tensors in this rank's order) and its context."""
    ctx: object
    x: object
    y: object
    z: object
    m: object
    vx: object = None
    vy: object = None
    vz: object = None
    gid: object = None
    info: dict = field(default_factory=dict)


def _global_counts(comm, parts, box):
    def fn(ranges):
        lo = [r[0] for r in ranges]
        hi = [r[1] for r in ranges]
        local = [np.array(p.ctx.key_range_counts(p.x, p.y, p.z, box, lo, hi), dtype=np.int64) for p in parts]
        return comm.allreduce(local, "sum")[0]
    return fn


def decompose(comm, parts, params):
    """Redistribute the ranks' particles by key range and build and join every
    rank's tree; afterwards p.ctx.far_force / neighbours / kick act on p's new
    particles (p.x, ... replaced, p.gid their global indices).  parts: one RankPart
    per rank of this process (comm.ranks)."""
    import torch
    P = comm.size
    # 1. the global bounding box (rule 1 on the whole cluster)
    boxes = [np.array(p.ctx.local_bbox(p.x, p.y, p.z)) if p.x.numel() > 0 else
             np.array([np.inf] * 3 + [-np.inf] * 3) for p in parts]
    lo = comm.allreduce([b[:3] for b in boxes], "min")[0]
    hi = comm.allreduce([b[3:] for b in boxes], "max")[0]
    gbox = [float(v) for v in lo] + [float(v) for v in hi]
    n_total = int(comm.allreduce([np.array([p.x.numel()], dtype=np.int64) for p in parts], "sum")[0][0])
    threshold = max(GROUP_NODE_FACTOR * params.group_size, params.leaf_cap)
    counts = _global_counts(comm, parts, gbox)
    # 2. splitters, then the particles to their ranks
    bounds = choose_splitters(n_total, P, threshold, counts)
    send = []
    for p in parts:
        arrays = [p.x, p.y, p.z, p.m] + ([p.vx, p.vy, p.vz] if p.vx is not None else []) + [p.gid]
        packed, cnt = p.ctx.partition(p.x, p.y, p.z, gbox, bounds, arrays)
        off = np.concatenate([[0], np.cumsum(cnt)])
        # one flat buffer per destination: the arrays' slices one after another (8-byte words)
        row = []
        for d in range(P):
            row.append(torch.cat([a[off[d]:off[d + 1]].view(torch.int64) for a in packed]))
        send.append(row)
    recv = comm.alltoall(send)
    has_v = parts[0].vx is not None
    na = 8 if has_v else 5
    for p, got in zip(parts, recv):
        cols = [[] for _ in range(na)]
        for buf in got:
            k = buf.numel() // na
            for a in range(na):
                cols[a].append(buf[a * k:(a + 1) * k])
        cat = [torch.cat(c) for c in cols]
        f64 = [c.view(torch.float64) for c in cat[:na - 1]]
        p.x, p.y, p.z, p.m = f64[:4]
        if has_v:
            p.vx, p.vy, p.vz = f64[4:7]
        p.gid = cat[-1]
    # 3. top cells, then every rank's tree
    tops = top_cells(bounds, _global_counts(comm, parts, gbox))
    for p in parts:
        p.ctx.build_tree_range(p.x, p.y, p.z, p.m, p.gid, gbox, [k for k, _ in tops], [l for _, l in tops])
    # 4. every rank's subtree boxes, locally essential trees, joins
    dom = comm.allgather([p.ctx.subtree_boxes() for p in parts])[0]
    r_halo = max(params.r_out, params.r_list)
    send_n, send_p, meta = [], [], []
    for i, p in enumerate(parts):
        me = comm.ranks[i]
        rn, rp, rm = [], [], []
        for d in range(P):
            if d == me:
                rn.append(torch.empty(0, dtype=torch.uint8, device=p.x.device))
                rp.append(torch.empty(0, dtype=torch.uint8, device=p.x.device))
                rm.append((0, 0, 0))
                continue
            nodes, pts, nn, nr, npt = p.ctx.let_export(dom[d], r_halo)
            rn.append(nodes[:nn * 288])
            rp.append(pts[:npt * 96])
            rm.append((nn, nr, npt))
        send_n.append(rn)
        send_p.append(rp)
        meta.append(rm)
    recv_n = comm.alltoall(send_n)
    recv_p = comm.alltoall(send_p)
    recv_m = comm.alltoall([[torch.tensor(m, dtype=torch.int64) for m in row] for row in meta])
    for i, p in enumerate(parts):
        me = comm.ranks[i]
        lets = []
        for s in range(P):
            if s == me:
                continue
            nn, nr, npt = (int(v) for v in recv_m[i][s].tolist())
            lets.append((recv_n[i][s], recv_p[i][s], nn, nr, npt))
        p.ctx.tree_join(lets)
        p.info = {"bounds": bounds, "top_cells": len(tops), "global_box": gbox,
                  "let_nodes_in": sum(l[2] for l in lets), "let_parts_in": sum(l[4] for l in lets)}
    return parts
