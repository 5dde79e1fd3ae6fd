"""Serving loop: distant-force steps for many device-resident clusters, with
continuous batching.

Clients ask for one step of a resident cluster (the step of the P3T scheme's
distant-force side: tree build, far force F_R of Eq. 3, neighbour lists of
Sec. 2.3, kick of Eq. 12, and the drift that stands in for the Hermite side).
Requests arrive at any time.  The server:

* admits them by device-memory footprint: it owns a fixed number of execution
  slots, each pre-sized (p3t_reserve plus staging buffers) for a budget of B
  particles, and a batch takes requests in arrival order while their particles
  fit in B -- so the device memory in use never grows while serving;
* batches continuously: whenever a slot is free and requests are waiting, it
  forms a batch from what has arrived and launches it on that slot's stream;
  requests that arrive while other batches run go into the next free slot, so
  the work of several batches overlaps on the device;
* keeps each cluster's steps in order: a cluster with a step in flight is not
  admitted again until that step completes.

A batch on a slot: gather its clusters from the arena into contiguous
staging (p3t_batch_move), one batched step (p3t_build_tree_batch with each
cluster's own theta / r_in / r_out / r_list, one persistent walk for all of
them, neighbour lists, kick, drift), scatter the state, accelerations and
cluster-local neighbour rows back (p3t_batch_move,
p3t_batch_scatter_neighbours), and an event marks completion.  Every kernel
is the library's; this module only schedules.

The scheduling policy (``Scheduler``) is plain host logic and is tested on the
CPU with a fake executor.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

# ---------------------------------------------------------------------------- policy


@dataclass
class Request:
    rid: int
    cluster: int
    t_arrival: float
    t_launch: float = math.nan
    t_done: float = math.nan
    batch: int = -1
    slot: int = -1


@dataclass
class Batch:
    bid: int
    slot: int
    requests: list
    particles: int


class Scheduler:
    """Admission and batching policy.

    sizes[k]: particles of cluster k; budget: particles per slot (the slot's
    memory footprint); max_clusters: segments per batch.  Requests are kept in
    arrival order.  ``form_batch`` walks the waiting requests oldest first and
    admits each whose cluster is idle and not yet in the batch, while the
    batch's particle total stays within the budget; it stops at the first
    idle-cluster request that does not fit (no overtaking, so no request
    starves).  A cluster larger than the budget can never run and is refused
    at submission.
    """

    def __init__(self, sizes, n_slots: int, budget: int, max_clusters: int = 256):
        if n_slots < 1 or budget < 1 or max_clusters < 1:
            raise ValueError("n_slots, budget and max_clusters must be positive")
        self.sizes = [int(s) for s in sizes]
        self.n_slots = n_slots
        self.budget = int(budget)
        self.max_clusters = int(max_clusters)
        self.waiting = collections.deque()
        self.busy_cluster = set()
        self.free_slots = list(range(n_slots))
        self.in_flight = {}
        self._bid = 0

    def submit(self, req: Request):
        if not 0 <= req.cluster < len(self.sizes):
            raise ValueError("unknown cluster %d" % req.cluster)
        if self.sizes[req.cluster] > self.budget:
            raise ValueError("cluster %d (%d particles) exceeds the slot budget %d"
                             % (req.cluster, self.sizes[req.cluster], self.budget))
        self.waiting.append(req)

    def form_batch(self):
        """A batch for a free slot, or None (no free slot, or nothing admissible)."""
        if not self.free_slots or not self.waiting:
            return None
        chosen, total, taken = [], 0, set()
        keep = collections.deque()
        blocked = False
        while self.waiting:
            r = self.waiting.popleft()
            if blocked or r.cluster in self.busy_cluster or r.cluster in taken \
                    or len(chosen) >= self.max_clusters:
                keep.append(r)
                continue
            n = self.sizes[r.cluster]
            if total + n > self.budget:
                blocked = True
                keep.append(r)
                continue
            chosen.append(r)
            taken.add(r.cluster)
            total += n
        self.waiting = keep
        if not chosen:
            return None
        slot = self.free_slots.pop(0)
        b = Batch(self._bid, slot, chosen, total)
        self._bid += 1
        for r in chosen:
            self.busy_cluster.add(r.cluster)
            r.batch, r.slot = b.bid, slot
        self.in_flight[b.bid] = b
        return b

    def complete(self, bid: int):
        b = self.in_flight.pop(bid)
        for r in b.requests:
            self.busy_cluster.discard(r.cluster)
        self.free_slots.append(b.slot)
        self.free_slots.sort()
        return b

    @property
    def idle(self) -> bool:
        return not self.waiting and not self.in_flight


def poisson_arrivals(rate: float, count: int, n_clusters: int, seed: int):
    """`count` requests with exponential gaps of mean 1/rate (seconds), each for a
    uniformly drawn cluster: [(t, cluster)], t ascending from 0."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    t -= t[0]
    cl = rng.integers(0, n_clusters, count)
    return [(float(a), int(b)) for a, b in zip(t, cl)]


def latency_stats(reqs):
    import numpy as np
    lat = np.array([r.t_done - r.t_arrival for r in reqs])
    wait = np.array([r.t_launch - r.t_arrival for r in reqs])
    return {"count": len(reqs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
            "max_ms": float(lat.max() * 1e3), "queue_wait_p50_ms": float(np.percentile(wait, 50) * 1e3),
            "queue_wait_p99_ms": float(np.percentile(wait, 99) * 1e3)}


# ---------------------------------------------------------------------------- device side


class Arena:
    """Resident clusters in device memory: FP64 state (x, y, z, m, vx, vy, vz), FP32
    accelerations, and cluster-local neighbour rows (n_k + 1 offsets and up to
    nbr_cap * n_k entries per cluster); plus each cluster's {theta, r_in, r_out,
    r_list}."""

    def __init__(self, clusters, params_rows, nbr_cap: int = 16, device=None):
        import numpy as np
        import torch
        self.torch = torch
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.sizes = [c.n for c in clusters]
        self.n_clusters = len(clusters)
        off = np.zeros(self.n_clusters + 1, np.int64)
        np.cumsum(self.sizes, out=off[1:])
        self.off = off
        self.total = int(off[-1])
        self.row_off = off[:-1] + np.arange(self.n_clusters)  # n_k + 1 offsets per cluster
        self.ent_cap = np.asarray(self.sizes, np.int64) * nbr_cap
        self.ent_off = np.concatenate([[0], np.cumsum(self.ent_cap)[:-1]]).astype(np.int64)
        self.params = np.asarray(params_rows, np.float64).reshape(self.n_clusters, 4)
        cat = lambda a: torch.from_numpy(np.ascontiguousarray(  # noqa: E731
            np.concatenate([getattr(c, a) for c in clusters]))).to(dev)
        self.state = {k: cat(k) for k in ("x", "y", "z", "m", "vx", "vy", "vz")}
        self.acc = [torch.zeros(self.total, dtype=torch.float32, device=dev) for _ in range(3)]
        self.nbr_offsets = torch.zeros(self.total + self.n_clusters, dtype=torch.int64, device=dev)
        self.nbr_idx = torch.zeros(int(self.ent_cap.sum()), dtype=torch.int32, device=dev)

    def cluster_view(self, k: int):
        """Views of cluster k's state, accelerations and neighbour rows (device tensors)."""
        s0, s1 = int(self.off[k]), int(self.off[k + 1])
        r0 = int(self.row_off[k])
        e0 = int(self.ent_off[k])
        out = {q: v[s0:s1] for q, v in self.state.items()}
        out["a"] = [a[s0:s1] for a in self.acc]
        out["offsets"] = self.nbr_offsets[r0:r0 + (s1 - s0) + 1]
        out["idx_base"] = self.nbr_idx[e0:e0 + int(self.ent_cap[k])]
        return out

    def bytes(self) -> int:
        return sum(v.numel() * v.element_size() for v in
                   list(self.state.values()) + self.acc + [self.nbr_offsets, self.nbr_idx])


class Slot:
    """One execution slot: a context on its own stream, pre-sized for `budget`
    particles in up to `max_clusters` clusters, with its staging buffers."""

    STAGING_BYTES_PER_PARTICLE = 7 * 8 + 3 * 4 + 8  # state, accelerations, row offsets (+ entries)

    def __init__(self, index, params, budget, max_clusters, nbr_cap, dt, device, lists_first=True):
        import torch

        import paper_2110_11658_b300 as p3t
        self.p3t = p3t
        self.torch = torch
        self.index = index
        self.dt = dt
        self.budget = budget
        self.max_clusters = max_clusters
        self.nbr_cap = nbr_cap
        self.stream = torch.cuda.Stream(device)
        self.ctx = p3t.Context(params, self.stream)
        self.ctx.reserve(budget, max_clusters)
        f64 = dict(dtype=torch.float64, device=device)
        self.st = {k: torch.zeros(budget, **f64) for k in ("x", "y", "z", "m", "vx", "vy", "vz")}
        self.acc = [torch.zeros(budget, dtype=torch.float32, device=device) for _ in range(3)]
        self.offs = torch.zeros(budget + 1, dtype=torch.int64, device=device)
        self.idx = torch.zeros(nbr_cap * budget, dtype=torch.int32, device=device)
        self.tot = torch.zeros(1, dtype=torch.int64, device=device)
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        i64 = dict(dtype=torch.int64)
        # host mirrors (pinned) and device copies of the batch description
        self.h_int = torch.zeros(5, max_clusters + 1, **i64).pin_memory()
        self.d_int = torch.zeros(5, max_clusters + 1, dtype=torch.int64, device=device)
        self.h_prm = torch.zeros(max_clusters, 4, dtype=torch.float64).pin_memory()
        self.d_prm = torch.zeros(max_clusters, 4, dtype=torch.float64, device=device)
        self.h_status = torch.zeros(1, dtype=torch.int32).pin_memory()
        self.done = torch.cuda.Event()
        self.batch = None
        self.sized = False  # the first batch's lists are synchronous: they size the row scratch
        # the lists before the far force: their own count pass, then a force-only walk
        # (faster for the short rows of the paper's r_cut; the same results)
        self.lists_first = lists_first

    def launch(self, arena: Arena, batch: Batch):
        import numpy as np
        torch = self.torch
        p3t = self.p3t
        ks = [r.cluster for r in batch.requests]
        c = len(ks)
        sizes = np.asarray([arena.sizes[k] for k in ks], np.int64)
        boff = np.zeros(c + 1, np.int64)
        np.cumsum(sizes, out=boff[1:])
        nb = int(boff[-1])
        h = self.h_int.numpy()
        h[0, :c + 1] = boff
        h[1, :c] = arena.off[ks]
        h[2, :c] = arena.row_off[ks]
        h[3, :c] = arena.ent_off[ks]
        h[4, :c] = arena.ent_cap[ks]
        self.h_prm.numpy()[:c] = arena.params[ks]
        s = self.stream
        with torch.cuda.stream(s):
            self.d_int.copy_(self.h_int, non_blocking=True)
            self.d_prm.copy_(self.h_prm, non_blocking=True)
            self.status.zero_()
        boff_d, aoff_d = self.d_int[0, :c + 1], self.d_int[1, :c]
        keys = ("x", "y", "z", "m", "vx", "vy", "vz")
        p3t.batch_move(s, c, nb, boff_d, aoff_d, [(arena.state[k], self.st[k]) for k in keys], True)
        st = {k: v[:nb] for k, v in self.st.items()}
        a = [v[:nb] for v in self.acc]
        ctx = self.ctx
        ctx.build_tree_batch(boff_d, st["x"], st["y"], st["z"], st["m"], cluster_params=self.d_prm[:c])
        if not self.lists_first:
            ctx.far_force(*a)
        if self.sized:
            ctx.neighbours_async(self.offs[:nb + 1], self.idx, self.tot)
        else:
            # once per slot (a host sync): sizes the row scratch, so that the
            # following batches' passes that count the neighbours also write their
            # rows (row mode)
            try:
                total = ctx.neighbours(self.offs[:nb + 1], self.idx)
            except p3t.P3TError as e:  # reported by the scatter's status, as in the async form
                if e.code != p3t.P3T_ERR_CAPACITY:
                    raise
                total = e.total
            with torch.cuda.stream(s):
                self.tot.fill_(total)
            self.sized = True
        if self.lists_first:
            ctx.far_force(*a)
        ctx.kick(self.dt, *a, st["vx"], st["vy"], st["vz"])
        ctx.drift(self.dt, st["x"], st["y"], st["z"], st["vx"], st["vy"], st["vz"])
        back = [(arena.state[k], self.st[k]) for k in ("x", "y", "z", "vx", "vy", "vz")]
        back += [(arena.acc[i], self.acc[i]) for i in range(3)]
        p3t.batch_move(s, c, nb, boff_d, aoff_d, back, False)
        p3t.batch_scatter_neighbours(s, c, nb, self.idx.numel(), boff_d, self.d_int[2, :c], self.d_int[3, :c],
                                     self.d_int[4, :c], self.offs, self.idx, arena.nbr_offsets, arena.nbr_idx,
                                     self.status)
        with torch.cuda.stream(s):
            self.h_status.copy_(self.status, non_blocking=True)
        self.done.record(s)
        self.batch = batch

    def ready(self) -> bool:
        return self.batch is not None and self.done.query()

    def finish(self):
        """Check the finished batch's status (the stream is idle up to its event)."""
        self.ctx.check()
        if int(self.h_status[0]) != 0:
            raise self.p3t.P3TError(int(self.h_status[0]), "serving batch %d" % self.batch.bid)
        b, self.batch = self.batch, None
        return b

    def close(self):
        self.ctx.close()


class Server:
    """Continuous-batching server over an Arena.

    n_slots execution slots of `budget` particles each (default: the largest
    cluster times `batch_factor`, capped by `hbm_budget` bytes over all slots);
    `max_clusters` segments per batch.  ``run(arrivals)`` replays a list of
    (t_seconds, cluster) arrivals in real time and returns the requests."""

    def __init__(self, arena: Arena, n_slots: int = 2, budget: int | None = None, max_clusters: int = 256,
                 nbr_cap: int = 16, dt: float = 1.0 / 512, leaf_cap: int = 16, group_size: int = 32,
                 tile: int = 64, hbm_budget: int | None = None, batch_factor: float = 8.0,
                 lists_first: bool = True):
        import paper_2110_11658_b300 as p3t
        self.arena = arena
        prm = p3t.Params(theta=float(arena.params[0, 0]), r_in=float(arena.params[0, 1]),
                         r_out=float(arena.params[0, 2]), r_list=float(arena.params[0, 3]), leaf_cap=leaf_cap,
                         group_size=group_size, tile=tile, precision=p3t.P3T_FP32_MIXED)
        biggest = max(arena.sizes)
        biggest = int(biggest)
        budget = int(biggest * batch_factor) if budget is None else int(budget)
        per_particle = (p3t.scratch_bytes(prm, budget, max_clusters) / budget
                        + Slot.STAGING_BYTES_PER_PARTICLE + 4 * nbr_cap)
        if hbm_budget is not None:
            budget = min(budget, int(hbm_budget / (n_slots * per_particle)))
        if budget < biggest:
            raise ValueError("the device-memory budget cannot hold the largest cluster")
        self.budget = budget
        self.bytes_per_slot = int(per_particle * budget)
        self.sched = Scheduler(arena.sizes, n_slots, budget, max_clusters)
        arena.torch.cuda.synchronize(arena.device)  # the arena was filled on another stream
        self.slots = [Slot(i, prm, budget, max_clusters, nbr_cap, dt, arena.device, lists_first)
                      for i in range(n_slots)]
        self.batches = []

    def close(self):
        for s in self.slots:
            s.close()

    def _pump(self, now_fn):
        progressed = False
        for s in self.slots:
            if s.ready():
                b = s.finish()
                t = now_fn()
                for r in b.requests:
                    r.t_done = t
                self.sched.complete(b.bid)
                progressed = True
        while True:
            b = self.sched.form_batch()
            if b is None:
                break
            t = now_fn()
            for r in b.requests:
                r.t_launch = t
            self.slots[b.slot].launch(self.arena, b)
            self.batches.append((b.bid, b.slot, len(b.requests), b.particles))
            progressed = True
        return progressed

    def run(self, arrivals, clock=time.perf_counter):
        """Replay arrivals [(t, cluster)] in real time; returns the completed requests."""
        reqs = [Request(i, c, t) for i, (t, c) in enumerate(arrivals)]
        t0 = clock()
        now = lambda: clock() - t0  # noqa: E731
        nxt = 0
        while nxt < len(reqs) or not self.sched.idle:
            t = now()
            while nxt < len(reqs) and reqs[nxt].t_arrival <= t:
                self.sched.submit(reqs[nxt])
                nxt += 1
            if not self._pump(now) and nxt < len(reqs):
                gap = reqs[nxt].t_arrival - now()
                if gap > 2e-4 and self.sched.idle:
                    time.sleep(gap - 1e-4)
        return reqs

    def run_serial(self, ks):
        """Run the steps of clusters ks one after another (each alone); for tests."""
        for k in ks:
            r = Request(-1, k, 0.0)
            self.sched.submit(r)
            b = self.sched.form_batch()
            assert b is not None and b.requests == [r]
            self.slots[b.slot].launch(self.arena, b)
            self.slots[b.slot].done.synchronize()
            self.slots[b.slot].finish()
            self.sched.complete(b.bid)


def summary(reqs, sizes, batches):
    """Latency percentiles, throughput and batch statistics of a finished run."""
    import numpy as np
    st = latency_stats(reqs)
    t_first = min(r.t_arrival for r in reqs)
    t_last = max(r.t_done for r in reqs)
    parts = sum(sizes[r.cluster] for r in reqs)
    st.update({"particles": int(parts), "span_s": t_last - t_first,
               "particles_per_s": parts / (t_last - t_first),
               "requests_per_s": len(reqs) / (t_last - t_first),
               "offered_requests_per_s": (len(reqs) - 1) / max(1e-12, max(r.t_arrival for r in reqs) - t_first)})
    if batches:
        nreq = np.array([b[2] for b in batches])
        npart = np.array([b[3] for b in batches])
        st.update({"batches": len(batches), "requests_per_batch_mean": float(nreq.mean()),
                   "requests_per_batch_max": int(nreq.max()), "particles_per_batch_mean": float(npart.mean())})
    return st
