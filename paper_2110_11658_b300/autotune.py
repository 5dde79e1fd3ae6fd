"""Autotuner of the walk's launch shape for a workload (ensemble or single cluster).

The tuned knobs are the walk group size G (targets that share one interaction
list), the threads per group (one warp with G/32 targets per lane, or G
threads in G/32 warps with one target each, the first warp walking the tree),
the list tile (interaction-list entries queued in shared memory before they
are evaluated) and the leaf capacity L of the octree.  G and L change the group and leaf boxes and so the
interaction lists themselves: a tuned configuration is part of the result's
identity, and the oracle reproduces a result given the same G and L.

The search runs in three stages to bound its cost: G x threads per group x tile
at the default leaf capacity, then L at the best (G, threads, tile), then the
order of a step's far force and neighbour lists at the best shape (the walk
counting the neighbours, or the lists' own count pass first and a force-only
walk: the second pays when the rows are short).  The threads per group and the
order change only how the same lists and forces are computed, not the results.
Every candidate is timed by a
caller-supplied function (normally a graph-captured step of the real
workload, see ``time_graph_step``) as the median of a few repeats.  Results
can be cached in a JSON file, keyed by a workload signature.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
from dataclasses import dataclass, field

GROUP_SIZES = (32, 64, 128)
TILES = (32, 64, 128, 256)
LEAF_CAPS = (8, 16, 32)
ORDERS = (0, 1)  # lists_first: the far force before the lists (0) or after them (1)
DEFAULT = {"group_size": 32, "threads_per_group": 32, "tile": 64, "leaf_cap": 16, "lists_first": 0}


def thread_counts(g: int):
    """Threads per group worth trying for G: one warp, or one thread per target."""
    return (32,) if g <= 32 else (32, 32 * ((g + 31) // 32))


def valid(cfg: dict) -> bool:
    """Launch shapes p3t_create accepts (tile a multiple of 32 in [32, 256], G <= 128,
    32, 64 or 128 threads per group with G <= threads beyond one warp)."""
    g, t, leaf = cfg["group_size"], cfg["tile"], cfg["leaf_cap"]
    tpg = cfg.get("threads_per_group", 32)
    return (1 <= g <= 128 and 32 <= t <= 256 and t % 32 == 0 and 1 <= leaf <= (1 << 20)
            and tpg in (32, 64, 128) and (tpg == 32 or g <= tpg) and cfg.get("lists_first", 0) in (0, 1))


def workload_key(device: str, sizes, precision: int, theta, extra: str = "") -> str:
    """Signature of a workload: device name, the cluster sizes, precision and theta."""
    h = hashlib.sha256(",".join(str(int(s)) for s in sizes).encode()).hexdigest()[:16]
    return "%s|C%d|N%d|%s|p%d|th%s|%s" % (device, len(sizes), int(sum(sizes)), h, precision,
                                        ",".join("%.4g" % t for t in (theta if hasattr(theta, "__len__") else [theta])),
                                        extra)


@dataclass
class Result:
    best: dict
    best_ms: float
    table: list = field(default_factory=list)  # [(cfg, ms)] in the order timed
    cached: bool = False


class Tuner:
    """Three-stage search over (G, threads per group, tile), then leaf capacity,
    then the order of far force and lists.

    time_fn(cfg) -> milliseconds of one step with that configuration; it is
    called `repeats` times per candidate and the median is kept.
    """

    def __init__(self, time_fn, repeats: int = 3, cache_path: str | None = None,
                 group_sizes=GROUP_SIZES, tiles=TILES, leaf_caps=LEAF_CAPS, orders=ORDERS):
        self.time_fn = time_fn
        self.repeats = max(1, int(repeats))
        self.cache_path = cache_path
        self.group_sizes, self.tiles, self.leaf_caps = tuple(group_sizes), tuple(tiles), tuple(leaf_caps)
        self.orders = tuple(orders)

    def _load(self) -> dict:
        if self.cache_path and os.path.exists(self.cache_path):
            with open(self.cache_path) as fh:
                return json.load(fh)
        return {}

    def _store(self, key: str, res: Result):
        if not self.cache_path:
            return
        data = self._load()
        data[key] = {"best": res.best, "best_ms": res.best_ms,
                     "table": [[c, ms] for c, ms in res.table]}
        tmp = self.cache_path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def _measure(self, cfg: dict) -> float:
        return statistics.median(float(self.time_fn(dict(cfg))) for _ in range(self.repeats))

    def tune(self, key: str | None = None) -> Result:
        if key is not None:
            hit = self._load().get(key)
            if hit is not None:
                return Result(hit["best"], hit["best_ms"], [(c, ms) for c, ms in hit["table"]], cached=True)
        table = []
        stage1 = [{"group_size": g, "threads_per_group": w, "tile": t, "leaf_cap": DEFAULT["leaf_cap"],
                   "lists_first": DEFAULT["lists_first"]}
                  for g in self.group_sizes for w in thread_counts(g) for t in self.tiles]
        for cfg in stage1:
            if valid(cfg):
                table.append((cfg, self._measure(cfg)))
        if not table:
            raise ValueError("no valid candidate")
        best, _ = min(table, key=lambda e: e[1])
        for leaf in self.leaf_caps:
            cfg = dict(best, leaf_cap=leaf)
            if valid(cfg) and all(cfg != c for c, _ in table):
                table.append((cfg, self._measure(cfg)))
        best, _ = min(table, key=lambda e: e[1])
        for order in self.orders:
            cfg = dict(best, lists_first=order)
            if valid(cfg) and all(cfg != c for c, _ in table):
                table.append((cfg, self._measure(cfg)))
        best, best_ms = min(table, key=lambda e: e[1])
        res = Result(dict(best), best_ms, table)
        if key is not None:
            self._store(key, res)
        return res


def time_graph_step(make_graph, steps: int = 3, flush_bytes: int = 256 << 20):
    """Build a time_fn from make_graph(cfg) -> (graph, ctx): one untimed launch,
    then `steps` launches each timed with CUDA events on the context's stream,
    the L2 flushed before each; returns the median in milliseconds."""
    import torch

    flush = torch.empty(flush_bytes, dtype=torch.uint8, device="cuda")

    def fn(cfg):
        graph, ctx = make_graph(cfg)
        try:
            graph.launch()
            ctx.check()
            s = ctx.stream
            ts = []
            for _ in range(steps):
                with torch.cuda.stream(s):
                    flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(s)
                graph.launch()
                e1.record(s)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ctx.check()
            return statistics.median(ts)
        finally:
            ctx.close()

    return fn
