"""Benchmark of the P3T distant-force path on one B300 (replicas on N GPUs).

Workload (the distant-force benchmark at N = 10^6): a Plummer sphere of
N = 1,000,000 stars with Kroupa masses (0.08-100, total mass 1) in Henon
units, theta = 0.4, monopole + quadrupole cells, r_out chosen for ~100 mean
neighbours (closed form 0.9006 N r^3 = 100 -> r_out = 0.0481), r_in =
0.1 r_out, r_list = r_out, FP32 interactions on FP64 relative coordinates.

One step = one pass of the whole path: tree build (keys, sort, topology,
moments, groups), far force, neighbour lists, kick (dt = 1/512) and the drift
x += dt v that stands in for the Hermite integration, so every step works on
moved particles.  Inputs are synthetic and seeded (data: "synthetic").

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the context's stream; between steps a 256 MB buffer is written to flush
the 126 MB L2 (outside the events).  The timed region is bracketed by a
barrier and a device synchronisation; the reported time is the maximum over
ranks.  value = particles processed by all ranks / time (far-force evals/s).

--impl reference runs the CPU oracle (plain FP64 C) on the same workload,
each step a bounded sample (see cpu_sample), on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# DRAM bytes (read + written) of one walk_kernel launch, from an ncu capture of the
# 10^6-particle Plummer walk of the timed step, which also writes the neighbour rows.
# Valid only at that N and for the kernel sources it was measured on (their hashes):
# otherwise the roofline's traffic is null.
WALK_TRAFFIC = {"sources": {"walk.cu": "9623c7c1f07c3515", "walk_f1.cu": "2881d95896a10898", "walk_kernel.cuh": "93d2e360329e8c2b", "p3t_internal.cuh": "1b7baccf169f4625"},
                "n": 1000000, "bytes": 302835968 + 506728192}

N_DEFAULT = 1_000_000
THETA = 0.4
DT = 1.0 / 512
FLOPS_PER_INTERACTION = 38
FP32_LANES_PER_SM = 128


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--group-size", type=int, default=32)
    ap.add_argument("--threads-per-group", type=int, default=32,
                    help="32: one warp per group; 64 or 128: one thread per target (G <= threads)")
    ap.add_argument("--tile", type=int, default=64)
    ap.add_argument("--leaf-cap", type=int, default=16)
    ap.add_argument("--r-buff", type=float, default=0.0,
                    help="neighbour buffer: r_list = r_out + r_buff (Eq. 20; 'paper' value 3 tau sigma "
                         "is passed as a negative number: -1 = one times the rule)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work")
    ap.add_argument("--ranks", type=int, default=2, help="decomp1m: virtual ranks on one GPU (without torchrun)")
    ap.add_argument("--workload", default="plummer1m",
                    choices=["plummer1m", "king2m", "ensemble64", "serve256", "irregular1m", "core1m", "decomp1m"],
                    help="plummer1m: the throughput benchmark; king2m: theta sweep of the "
                         "mixed and FP64 forms against the direct sum (one line per theta); "
                         "ensemble64: 64 clusters in one graph-captured batched step, autotuned, "
                         "against one-cluster-at-a-time launches; serve256: Poisson request stream over "
                         "256 resident clusters with continuous batching (p50/p99 latency); "
                         "irregular1m: irregular force and jerk over the neighbour rows of plummer1m; "
                         "core1m: 6 nearest neighbours of sqrt(5000 N) sampled particles and core quantities; "
                         "decomp1m: plummer1m decomposed over ranks (locally essential trees)")
    ap.add_argument("--requests", type=int, default=10000, help="serve256: requests in the timed stream")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve256: mean arrival rate (requests/s)")
    ap.add_argument("--no-tune", action="store_true", help="ensemble64: use --group-size/--tile/--leaf-cap")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="plummer1m: leave out the short ensemble64 summary (p50/p99) of the line")
    ap.add_argument("--ens-steps", type=int, default=20, help="timed steps of the short ensemble summary")
    ap.add_argument("--samples", type=int, default=8192, help="direct-sum targets (king2m)")
    return ap.parse_args(argv)


def workload(n, seed):
    import synth
    c = synth.plummer(n, seed, masses="kroupa")
    r_out = synth.plummer_r_for_mean_neighbours(n, 100.0)
    return c, {"theta": THETA, "r_out": r_out, "r_in": 0.1 * r_out, "r_list": r_out}


# ---------------------------------------------------------------------------- distributed
def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("P3T_BENCH_BACKEND", "nccl")
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, local, world


def dist_barrier(world, device=None):
    if world > 1:
        import torch.distributed as dist
        if device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def dist_max(value, world, device=None):
    """Maximum of a float over ranks (identity for one rank)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(value, world, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------- peaks
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def walk_traffic(n):
    import hashlib
    csrc = os.path.join(ROOT, "paper_2110_11658_b300", "csrc")
    for name, want in WALK_TRAFFIC["sources"].items():
        with open(os.path.join(csrc, name), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest()[:16] != want:
                return None
    return WALK_TRAFFIC["bytes"] if n == WALK_TRAFFIC["n"] else None


def fp32_peak_tflops(sm_count, sm_max_mhz):
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 flops (FMA) x max SM clock."""
    return sm_count * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------- CPU oracle
def cpu_sample(c, prm, budget_s, with_neighbours=True, group_size=32, leaf_cap=16):
    """Time the oracle on a bounded sample of one step; returns step-time estimate.

    The oracle builds the whole tree (all N particles), then evaluates the far
    force (and the neighbour lists) for the first groups of the tree until
    `budget_s` is spent, and kicks all particles.  The per-particle force and
    neighbour cost of the sample is scaled to all N.
    """
    import numpy as np

    import oracle
    t0 = time.perf_counter()
    tree = oracle.Tree(c.x, c.y, c.z, c.m, prm["theta"], prm["r_out"], leaf_cap=leaf_cap,
                       group_size=group_size)
    t_build = time.perf_counter() - t0
    ex = tree.export()
    gcount = ex["g_count"]
    ng = tree.n_groups
    done, t_force, t_nbr, parts = 0, 0.0, 0.0, 0
    chunk = max(1, ng // 1000)
    while done < ng and t_build + t_force + t_nbr < budget_s:
        sel = np.arange(done, min(ng, done + chunk))
        t1 = time.perf_counter()
        tree.far(prm["r_in"], groups=sel)
        t2 = time.perf_counter()
        if with_neighbours:
            tree.neighbours(prm["r_list"], groups=sel)
        t3 = time.perf_counter()
        t_force += t2 - t1
        t_nbr += t3 - t2
        parts += int(gcount[sel].sum())
        done += len(sel)
        chunk *= 2
    t4 = time.perf_counter()
    zeros = np.zeros(c.n)
    oracle.kick(DT, zeros, zeros, zeros, c.vx, c.vy, c.vz)
    t_kick = time.perf_counter() - t4
    scale = c.n / max(1, parts)
    step = t_build + (t_force + t_nbr) * scale + t_kick
    return {"step_s": step, "far_s_per_particle": t_force / max(1, parts), "sampled_particles": parts,
            "groups": int(done), "build_s": t_build, "wall_s": time.perf_counter() - t0}


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    if v and v.isdigit():
        return int(v)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------- GPU arm
def run_b300(args, rank, local, world):
    import numpy as np
    import torch

    import paper_2110_11658_b300 as p3t

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    c, w = workload(args.n, 20211022 + rank)
    if args.r_buff != 0.0:
        import synth
        rb = args.r_buff if args.r_buff > 0 else -args.r_buff * synth.paper_run_params(args.n)["r_buff"]
        w["r_list"] = w["r_out"] + rb
    prm = p3t.Params(theta=w["theta"], r_in=w["r_in"], r_out=w["r_out"], r_list=w["r_list"],
                     leaf_cap=args.leaf_cap, group_size=args.group_size, tile=args.tile,
                     threads_per_group=args.threads_per_group, precision=p3t.P3T_FP32_MIXED, quadrupole=1)
    stream = torch.cuda.current_stream(dev)
    ctx = p3t.Context(prm, stream)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    x, y, z, m = t(c.x), t(c.y), t(c.z), t(c.m)
    vx, vy, vz = t(c.vx), t(c.vy), t(c.vz)
    n = c.n
    a = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3)]
    offs = torch.empty(n + 1, dtype=torch.int64, device=dev)
    tot_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    n_cell = torch.zeros(1, dtype=torch.int64, device=dev)
    n_part = torch.zeros(1, dtype=torch.int64, device=dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)

    # size the neighbour buffer from one synchronous step
    ctx.build_tree(x, y, z, m)
    ctx.far_force(*a)
    try:
        ctx.neighbours(offs, torch.empty(1, dtype=torch.int32, device=dev))
        first_total = 0
    except p3t.P3TError as e:
        if e.code != p3t.P3T_ERR_CAPACITY:
            raise
        first_total = e.total
    idx = torch.empty(int(first_total * 1.3) + 1024, dtype=torch.int32, device=dev)

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(record):
        e0, e1, e2, e3, e4 = (ev(), ev(), ev(), ev(), ev()) if record else (None,) * 5
        if record:
            e0.record(stream)
        ctx.build_tree(x, y, z, m)
        if record:
            e1.record(stream)
        ctx.far_force(*a, n_cell=n_cell, n_part=n_part)
        if record:
            e2.record(stream)
        ctx.neighbours_async(offs, idx, tot_dev)
        if record:
            e3.record(stream)
        ctx.kick(DT, *a, vx, vy, vz)
        ctx.drift(DT, x, y, z, vx, vy, vz)
        if record:
            e4.record(stream)
        return (e0, e1, e2, e3, e4)

    for _ in range(max(3, args.warmup)):
        step(False)
    ctx.check()
    # the timed steps are CUDA-graph launches, one graph per step so that each has
    # its own phase events (event nodes inside the graph)
    graphs, evs = [], []
    for _ in range(args.steps):
        e5 = tuple(ev() for _ in range(5))
        graphs.append(ctx.capture_step(x, y, z, m, *a, vx=vx, vy=vy, vz=vz, kick_dt=DT, drift_dt=DT,
                                       n_cell=n_cell, n_part=n_part, offsets=offs, idx=idx, total=tot_dev,
                                       events=e5))
        evs.append(e5)
    n_cell.zero_()
    n_part.zero_()
    torch.cuda.synchronize(dev)
    dist_barrier(world, dev)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    wall0 = time.perf_counter()
    for g in graphs:
        flush.fill_(1)
        g.launch()
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    dist_barrier(world, dev)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    st = ctx.status()
    if st != p3t.P3T_OK:
        raise p3t.P3TError(st, "benchmark step")
    row_cap, rows_valid = ctx.row_mode()
    # the same walk without neighbour work (the lists built first, so the walk
    # neither counts nor writes rows): the kernel's force efficiency on its own
    fo = []
    for _ in range(6):
        flush.fill_(1)
        ctx.build_tree(x, y, z, m)
        ctx.neighbours_async(offs, idx, tot_dev)
        f0, f1 = ev(), ev()
        f0.record(stream)
        ctx.far_force(*a)
        f1.record(stream)
        fo.append((f0, f1))
    torch.cuda.synchronize(dev)
    far_only_ms = dist_max(statistics.median(f0.elapsed_time(f1) for f0, f1 in fo[1:]), world, dev)
    ph = {"build": 0.0, "far": 0.0, "nbr": 0.0, "kick_drift": 0.0}
    for e0, e1, e2, e3, e4 in evs:
        ph["build"] += e0.elapsed_time(e1)
        ph["far"] += e1.elapsed_time(e2)
        ph["nbr"] += e2.elapsed_time(e3)
        ph["kick_drift"] += e3.elapsed_time(e4)
    per_step = sorted(e0.elapsed_time(e4) for e0, e1, e2, e3, e4 in evs)
    step_ms_local = sum(ph.values()) / args.steps
    step_ms = dist_max(step_ms_local, world, dev)
    far_ms = dist_max(ph["far"] / args.steps, world, dev)
    ncell = int(n_cell.item()) / args.steps
    npart = int(n_part.item()) / args.steps
    inter = ncell + npart
    nbr_total = int(tot_dev.item())
    props = torch.cuda.get_device_properties(dev)
    peaks, peak_kind = measured_peaks()
    fp32_peak = fp32_peak_tflops(props.multi_processor_count, float(peaks.get("sm_max_mhz", 2032.0)))
    achieved = FLOPS_PER_INTERACTION * inter / (far_ms * 1e-3) / 1e12
    total_particles = dist_sum(float(n), world, dev)
    value = total_particles / (step_ms * 1e-3)

    # end-to-end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        pin = lambda q: torch.from_numpy(np.ascontiguousarray(q)).pin_memory()  # noqa: E731
        hx, hy, hz, hm = pin(c.x), pin(c.y), pin(c.z), pin(c.m)
        hv = [pin(c.vx), pin(c.vy), pin(c.vz)]
        ha = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(3)]
        hoffs = torch.empty(n + 1, dtype=torch.int64).pin_memory()
        hidx = torch.empty(idx.numel(), dtype=torch.int32).pin_memory()
        hctx = p3t.Context(prm, stream)
        for _ in range(2):
            hctx.step_host(DT, hx, hy, hz, hm, *hv, *ha, hoffs, hidx)
        k = max(3, min(args.steps, 10))
        dist_barrier(world, dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        tots = 0
        for _ in range(k):
            tots = hctx.step_host(DT, hx, hy, hz, hm, *hv, *ha, hoffs, hidx)
        torch.cuda.synchronize(dev)
        te = dist_max((time.perf_counter() - t0) / k, world, dev)
        hctx.close()
        e2e = {"value": total_particles / te, "unit": "particles/s",
               "h2d_bytes_per_step": 7 * 8 * n, "d2h_bytes_per_step": 3 * 4 * n + 3 * 8 * n + 8 * (n + 1) + 4 * tots,
               "ms_per_step": te * 1e3, "api": "p3t_step_host (pinned host buffers)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = cpu_sample(c, w, args.cpu_budget, group_size=args.group_size, leaf_cap=args.leaf_cap)
        cpu = {"value": c.n / s["step_s"], "unit": "particles/s", "cores": omp_threads(), "kind": "oracle",
               "sample": "oracle tree build of all %d particles, far force + neighbour lists of the first %d "
                         "groups (%d particles) scaled to all N, kick of all N; %.1f s of CPU work"
                         % (c.n, s["groups"], s["sampled_particles"], s["wall_s"]),
               "far_force_evals_per_s": 1.0 / s["far_s_per_particle"]}

    line = {
        "metric": "particle far-force evals/sec & interactions/sec at N=1e6 (FP32 % peak); ensemble p50/p99",
        "value": value,
        "unit": "particles/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(n, w, args, world),
        "precision": "fp32 interactions, fp64 coordinates, compensated sums",
        "step": "build_tree + far_force + neighbours + kick + drift, one CUDA graph launch",
        "far_force_evals_per_s": total_particles / (far_ms * 1e-3),
        "interactions_per_s": inter / (far_ms * 1e-3) * world,
        "interactions_per_particle": inter / n,
        "cell_interactions_per_particle": ncell / n,
        "particle_interactions_per_particle": npart / n,
        "fp32_pct_of_peak": 100.0 * achieved / fp32_peak,
        "phase_ms": {k: v / args.steps for k, v in ph.items()},
        "step_ms_p50": statistics.median(per_step),
        "step_ms_p99": per_step[min(len(per_step) - 1, int(round(0.99 * (len(per_step) - 1))))],
        "mean_neighbours": nbr_total / n,
        "roofline": {"bound": "alu", "kernel": "walk_kernel (p3t_far_force, counting and writing the "
                                              "neighbour rows)", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": walk_traffic(n),
                     "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x %.0f MHz (%s sm_max_mhz)"
                                    % (float(peaks.get("sm_max_mhz", 2032.0)), peak_kind),
                     "flops_per_launch": FLOPS_PER_INTERACTION * inter},
        "roofline_cells_only": {"note": "the cell (monopole + quadrupole) terms alone at 38 flops each over "
                                        "the same timed walk; the particle terms (W-weighted pairs) left out",
                                "achieved": FLOPS_PER_INTERACTION * ncell / (far_ms * 1e-3) / 1e12,
                                "frac": FLOPS_PER_INTERACTION * ncell / (far_ms * 1e-3) / 1e12 / fp32_peak},
        "roofline_force_only": {"kernel": "walk_kernel after the lists (no neighbour counting or rows)",
                                "far_ms": far_only_ms,
                                "achieved": FLOPS_PER_INTERACTION * inter / (far_only_ms * 1e-3) / 1e12,
                                "frac": FLOPS_PER_INTERACTION * inter / (far_only_ms * 1e-3) / 1e12 / fp32_peak},
        "neighbour_rows": {"written_by_walk": bool(rows_valid), "row_cap": row_cap},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * KERNELS_PER_STEP,
        "clocks": clk,
        "wall_s_timed": wall,
    }
    ctx.close()
    if rank == 0 and world == 1 and not args.no_ensemble:
        # the metric's ensemble p50/p99: the 64-cluster batched step, a few graph launches
        del x, y, z, m, vx, vy, vz, a, offs, idx, flush
        torch.cuda.empty_cache()
        line["ensemble"] = ensemble_run(args, short=True)
    return line


def bench_config(n, w, args, world):
    """The workload of the throughput line, identical in both arms."""
    return {"workload": "plummer_kroupa_n%d_theta%.1f_nbr100" % (n, THETA), "n": n, "theta": THETA,
            "r_out": w["r_out"], "r_in": w["r_in"], "r_list": w["r_list"], "leaf_cap": args.leaf_cap,
            "group_size": args.group_size, "threads_per_group": args.threads_per_group, "tile": args.tile,
            "dt": DT, "quadrupole": True,
            "l2": "256 MB buffer written between timed steps (L2 is 126 MB)",
            "parallelism": "replicas" if world > 1 else "single"}


# kernels launched by one step: build = metadata, cluster table, cluster parameters,
# bbox, cube, keys (6) + radix sort 8 x (histogram, scan, scatter) + gather + topology
# (per-particle levels, their scan, level table, nodes, counts and children) + group
# scan, first, finish, frames, walk order (bins, scan, scatter) + moments leaves and 21
# levels; far force 5 (the rows' layout from the last counts and its scan, the
# cell-form flags, then the walk in its two cell forms, one of which returns at once;
# the walk also counts the neighbours and writes the rows); neighbours = offsets scan,
# fill, row binning by length (count, list) and nine row-sort size classes; kick 1;
# drift 1 (85, as the ncu launch list of the step shows)
KERNELS_PER_STEP = (6 + 8 * 3 + 1 + 5 + 4 + 3 + (1 + 21)) + 5 + (2 + 2 + 9) + 1 + 1


def run_reference(args, rank, world):
    if rank != 0:
        return None
    c, w = workload(args.n, 20211022)
    times = []
    samples = []
    for i in range(args.warmup + args.steps):
        s = cpu_sample(c, w, max(2.0, args.cpu_budget / 4), group_size=args.group_size,
                       leaf_cap=args.leaf_cap)
        if i >= args.warmup:
            times.append(s["step_s"])
            samples.append(s)
    step = statistics.mean(times)
    value = c.n / step
    cores = omp_threads()
    sample = ("per step: oracle tree build of all %d particles, far force + neighbour lists of the first "
              "~%d particles' groups scaled to all N, kick of all N" % (c.n, samples[-1]["sampled_particles"]))
    return {
        "impl": "reference",
        "metric": "particle far-force evals/sec & interactions/sec at N=1e6 (FP32 % peak); ensemble p50/p99",
        "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": bench_config(c.n, w, args, world),
        "precision": "fp64 throughout (the oracle)",
        "step": "oracle tree build + far force + neighbour lists + kick, a bounded sample scaled to N",
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def king2m_sweep(args):
    """King W0 = 7, N = 2^21, Kroupa masses, heavy stars scaled by 0.7 (segregated);
    r_out = the paper's r_cut = 4 tau (Eqs. 21-22), r_in = 0.1 r_out.  For theta in
    {0.3, 0.5, 0.7}: far-force time of the mixed and all-FP64 GPU forms and their error
    against the FP64 direct sum on `samples` seeded targets."""
    import numpy as np
    import torch

    import oracle
    import paper_2110_11658_b300 as p3t
    import synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n = 2 ** 21 if args.n == N_DEFAULT else args.n
    c = synth.make("king", n, 20211022, masses="kroupa", w0=7.0, segregated=True)
    r_out = synth.paper_run_params(n)["r_cut"]
    r_in = 0.1 * r_out
    tg = np.random.default_rng(20211022).choice(n, args.samples, replace=False)
    t0 = time.perf_counter()
    ref = oracle.direct_split(c.x, c.y, c.z, c.m, r_in, r_out, targets=tg)["far"]
    t_direct = time.perf_counter() - t0
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    x, y, z, m = t(c.x), t(c.y), t(c.z), t(c.m)
    lines = []
    for theta in (0.3, 0.5, 0.7):
        row = {"theta": theta}
        for name, prec in (("mixed", p3t.P3T_FP32_MIXED), ("fp64", p3t.P3T_FP64)):
            prm = p3t.Params(theta=theta, r_in=r_in, r_out=r_out, r_list=r_out, leaf_cap=args.leaf_cap,
                             group_size=args.group_size, tile=args.tile, precision=prec)
            ctx = p3t.Context(prm)
            ctx.build_tree(x, y, z, m)
            dt = ctx.acc_dtype
            a = [torch.empty(n, dtype=dt, device=dev) for _ in range(3)]
            nc = torch.zeros(1, dtype=torch.int64, device=dev)
            npart = torch.zeros(1, dtype=torch.int64, device=dev)
            reps = 5 if prec == p3t.P3T_FP32_MIXED else 2
            times = []
            for r in range(reps + 1):
                nc.zero_()
                npart.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.far_force(*a, n_cell=nc, n_part=npart)
                e1.record()
                torch.cuda.synchronize()
                if r:
                    times.append(e0.elapsed_time(e1))
            ctx.check()
            got = torch.stack(a, 1).double().cpu().numpy()[tg]
            err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
            inter = (int(nc.item()) + int(npart.item())) / n
            ms = float(np.median(times))
            row[name] = {"far_ms": ms, "evals_per_s": n / (ms * 1e-3),
                         "err_vs_direct_median": float(np.median(err)),
                         "err_vs_direct_p99": float(np.percentile(err, 99)),
                         "interactions_per_particle": inter}
            ctx.close()
        row["speedup_mixed_over_fp64"] = row["fp64"]["far_ms"] / row["mixed"]["far_ms"]
        lines.append(row)
    for row in lines:
        print(json.dumps({"workload": "king_w0_7_kroupa_segregated_n%d" % n, "n": n, "r_out": r_out,
                          "r_in": r_in, "samples": args.samples, "direct_sum_s": t_direct, **row}))


# ---------------------------------------------------------------------------- ensemble
ENS_CLUSTERS, ENS_N_LO, ENS_N_HI, ENS_THETA = 64, 1e4, 5e5, 0.4


def ensemble_params(sizes):
    """Per-cluster {theta, r_in, r_out, r_list}: r_out = the paper's r_cut = 4 tau(N)
    (Eqs. 21-22) of each cluster, r_in = 0.1 r_out, r_list = r_out."""
    import synth
    rows = []
    for n in sizes:
        rc = synth.paper_run_params(int(n))["r_cut"]
        rows.append([ENS_THETA, 0.1 * rc, rc, rc])
    return rows


def _events_ms(stream, fn, steps, flush):
    import torch
    ts = []
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts


def _dist(ts):
    import numpy as np
    a = np.asarray(ts)
    return {"mean": float(a.mean()), "p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)),
            "min": float(a.min()), "max": float(a.max()), "steps": len(ts)}


# the launch shape the autotuner picks for this ensemble (G, threads per group, list tile, leaf
# capacity, and the lists before the far force)
ENS_TUNED = {"group_size": 32, "threads_per_group": 32, "tile": 64, "leaf_cap": 16, "lists_first": 1}


def ensemble_run(args, short=False):
    """64 independent clusters (alternately Plummer and King W0 = 5), N log-uniform in
    [1e4, 5e5] (~7.8e6 in total), equal masses, theta = 0.4, per-cluster r_out by the
    paper's rule.  One step = batched build + far force + neighbour lists + kick + drift,
    captured once into a CUDA graph (one persistent walk launch for every cluster), with
    the launch shape picked by the autotuner.  Compared with the same step run one
    cluster at a time (eager calls, and one graph per cluster).

    short: the summary the throughput benchmark attaches to its line: the tuned shape
    (ENS_TUNED) without a search, `args.ens_steps` timed steps of the batched graph and of
    one graph per cluster, no eager forms."""
    import numpy as np
    import torch

    import paper_2110_11658_b300 as p3t
    import synth
    from paper_2110_11658_b300 import autotune

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    cl = synth.ensemble(ENS_CLUSTERS, ENS_N_LO, ENS_N_HI, 20211022, masses="equal", w0=5.0)
    sizes = [c.n for c in cl]
    allc, segn = synth.concat(cl)
    n = allc.n
    rows = ensemble_params(sizes)
    stream = torch.cuda.Stream(dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    init = {k: t(getattr(allc, k)) for k in ("x", "y", "z", "m", "vx", "vy", "vz")}
    seg = t(segn)
    cprm = torch.tensor(rows, dtype=torch.float64, device=dev)
    cap = 16 * n
    buf = {"a": [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3)],
           "offs": torch.empty(n + 1, dtype=torch.int64, device=dev),
           "idx": torch.empty(cap, dtype=torch.int32, device=dev),
           "tot": torch.zeros(1, dtype=torch.int64, device=dev),
           "nc": torch.zeros(1, dtype=torch.int64, device=dev),
           "np": torch.zeros(1, dtype=torch.int64, device=dev)}
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)

    def params(cfg):
        return p3t.Params(theta=ENS_THETA, r_in=rows[0][1], r_out=rows[0][2], r_list=rows[0][3],
                          leaf_cap=cfg["leaf_cap"], group_size=cfg["group_size"], tile=cfg["tile"],
                          threads_per_group=cfg.get("threads_per_group", 32), precision=p3t.P3T_FP32_MIXED)

    def batched_graph(cfg, st):
        ctx = p3t.Context(params(cfg), stream)
        # one synchronous list first, as in the single-cluster step: it sizes the
        # row scratch, so the captured walks write the neighbour rows (row mode)
        ctx.build_tree_batch(seg, st["x"], st["y"], st["z"], st["m"], cluster_params=cprm)
        ctx.far_force(*buf["a"])
        ctx.neighbours(buf["offs"], buf["idx"])
        g = ctx.capture_step(st["x"], st["y"], st["z"], st["m"], *buf["a"], seg_offsets=seg, cluster_params=cprm,
                             vx=st["vx"], vy=st["vy"], vz=st["vz"], kick_dt=DT, drift_dt=DT,
                             n_cell=buf["nc"], n_part=buf["np"], offsets=buf["offs"], idx=buf["idx"],
                             total=buf["tot"], lists_first=bool(cfg.get("lists_first", 0)))
        return g, ctx

    tune_state = {k: v.clone() for k, v in init.items()}
    if short:
        best, table = dict(ENS_TUNED), []
    elif args.no_tune:
        best = {"group_size": args.group_size, "threads_per_group": args.threads_per_group, "tile": args.tile,
                "leaf_cap": args.leaf_cap, "lists_first": 0}
        table = []
    else:
        res = autotune.Tuner(autotune.time_graph_step(lambda cfg: batched_graph(cfg, tune_state), steps=3),
                             repeats=1).tune()
        best, table = res.best, [{"cfg": c, "ms": ms} for c, ms in res.table]
    del tune_state

    steps = max(3, args.ens_steps if short else args.steps)
    out = {}
    # (a) batched, graph-captured
    st = {k: v.clone() for k, v in init.items()}
    g, ctx = batched_graph(best, st)
    for _ in range(max(3, args.warmup)):
        g.launch()
    ctx.check()
    buf["nc"].zero_()
    buf["np"].zero_()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(0)
    clocks.start()
    out["batched_graph"] = _dist(_events_ms(stream, g.launch, steps, flush))
    clk = clocks.stop()
    ctx.check()
    inter = (int(buf["nc"].item()) + int(buf["np"].item())) / steps
    nbr_total = int(buf["tot"].item())
    row_cap, rows_valid = ctx.row_mode()
    # far force alone (eager, same context and tree) for the walk's roofline
    far_ts = _events_ms(stream, lambda: ctx.far_force(*buf["a"]), steps, flush)
    ctx.check()
    ctx.close()
    if short:
        del g
        per_s = _sequential_graph_ms(cl, segn, rows, init, buf, params(best), stream, dev, steps, flush,
                                     bool(best.get("lists_first", 0)))
        b = out["batched_graph"]
        return {"workload": "ensemble64_plummer_king5_n1e4-5e5", "n_clusters": len(cl), "particles": n,
                "shape": best, "steps": steps, "step_ms_p50": b["p50"], "step_ms_p99": b["p99"],
                "step_ms_mean": b["mean"], "particles_per_s": n / (b["mean"] * 1e-3),
                "one_cluster_at_a_time_ms_mean": per_s["mean"], "one_cluster_at_a_time_ms_p99": per_s["p99"],
                "speedup_vs_one_at_a_time": per_s["mean"] / b["mean"],
                "far_ms": float(np.median(far_ts)), "interactions_per_particle": inter / n,
                "step": "batched build + far force + neighbours + kick + drift, one CUDA graph launch; "
                        "one at a time = one graph per cluster, 64 launches",
                "clocks": clk}
    # (b) batched, eager calls
    st = {k: v.clone() for k, v in init.items()}
    ctx = p3t.Context(params(best), stream)

    lists_first = bool(best.get("lists_first", 0))

    def eager():
        ctx.build_tree_batch(seg, st["x"], st["y"], st["z"], st["m"], cluster_params=cprm)
        if lists_first:
            ctx.neighbours_async(buf["offs"], buf["idx"], buf["tot"])
            ctx.far_force(*buf["a"])
        else:
            ctx.far_force(*buf["a"])
            ctx.neighbours_async(buf["offs"], buf["idx"], buf["tot"])
        ctx.kick(DT, *buf["a"], st["vx"], st["vy"], st["vz"])
        ctx.drift(DT, st["x"], st["y"], st["z"], st["vx"], st["vy"], st["vz"])

    ctx.build_tree_batch(seg, st["x"], st["y"], st["z"], st["m"], cluster_params=cprm)
    ctx.far_force(*buf["a"])
    ctx.neighbours(buf["offs"], buf["idx"])  # sizes the row scratch (row mode)
    for _ in range(2):
        eager()
    out["batched_eager"] = _dist(_events_ms(stream, eager, steps, flush))
    ctx.check()
    ctx.close()
    # (c), (d) one cluster at a time: a context per cluster with its own r_out
    st = {k: v.clone() for k, v in init.items()}
    per = []
    for k, c in enumerate(cl):
        s0, s1 = int(segn[k]), int(segn[k + 1])
        prm = params(best)
        prm.r_in, prm.r_out, prm.r_list = rows[k][1], rows[k][2], rows[k][3]
        cx = p3t.Context(prm, stream)
        v = {q: st[q][s0:s1] for q in st}
        a = [buf["a"][i][s0:s1] for i in range(3)]
        offs = torch.empty(c.n + 1, dtype=torch.int64, device=dev)
        idx = buf["idx"][16 * s0:16 * s1]
        tot = torch.zeros(1, dtype=torch.int64, device=dev)
        cx.build_tree(v["x"], v["y"], v["z"], v["m"])
        cx.far_force(*a)
        cx.neighbours(offs, idx)  # sizes the row scratch (row mode)
        per.append((cx, v, a, offs, idx, tot))

    def sequential():
        for cx, v, a, offs, idx, tot in per:
            cx.build_tree(v["x"], v["y"], v["z"], v["m"])
            if lists_first:
                cx.neighbours_async(offs, idx, tot)
                cx.far_force(*a)
            else:
                cx.far_force(*a)
                cx.neighbours_async(offs, idx, tot)
            cx.kick(DT, *a, v["vx"], v["vy"], v["vz"])
            cx.drift(DT, v["x"], v["y"], v["z"], v["vx"], v["vy"], v["vz"])

    for _ in range(2):
        sequential()
    out["sequential_eager"] = _dist(_events_ms(stream, sequential, steps, flush))
    graphs = [cx.capture_step(v["x"], v["y"], v["z"], v["m"], *a, vx=v["vx"], vy=v["vy"], vz=v["vz"],
                              kick_dt=DT, drift_dt=DT, offsets=offs, idx=idx, total=tot, lists_first=lists_first)
              for cx, v, a, offs, idx, tot in per]

    def sequential_graphs():
        for gg in graphs:
            gg.launch()

    for _ in range(2):
        sequential_graphs()
    out["sequential_graph"] = _dist(_events_ms(stream, sequential_graphs, steps, flush))
    for cx, *_ in per:
        cx.check()
        cx.close()

    props = torch.cuda.get_device_properties(dev)
    peaks, peak_kind = measured_peaks()
    fp32_peak = fp32_peak_tflops(props.multi_processor_count, float(peaks.get("sm_max_mhz", 2032.0)))
    far_ms = float(np.median(far_ts))
    achieved = FLOPS_PER_INTERACTION * inter / (far_ms * 1e-3) / 1e12
    step_ms = out["batched_graph"]["mean"]
    return {
        "metric": "particle far-force evals/sec & interactions/sec at N=1e6 (FP32 % peak); ensemble p50/p99",
        "value": n / (step_ms * 1e-3), "unit": "particles/s", "n_gpus": 1, "steps": steps,
        "warmup": max(3, args.warmup), "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ensemble64_plummer_king5_n1e4-5e5", "n_clusters": len(cl), "n": n,
                   "sizes": sizes, "theta": ENS_THETA, "r_out": "paper r_cut = 4 tau(N) per cluster",
                   "r_in": "0.1 r_out", "r_list": "r_out", "dt": DT, "tuned": best,
                   "step": "batched build + far force + neighbours + kick + drift, one CUDA graph launch",
                   "l2": "256 MB buffer written between timed steps (L2 is 126 MB)"},
        "ensemble": {"step_ms": out, "speedup_vs_sequential_eager":
                     out["sequential_eager"]["mean"] / step_ms,
                     "speedup_vs_sequential_graph": out["sequential_graph"]["mean"] / step_ms,
                     "tuner_table": table},
        "far_ms": far_ms, "interactions_per_particle": inter / n, "mean_neighbours": nbr_total / n,
        "neighbour_rows": {"written_by_walk": bool(rows_valid), "row_cap": row_cap},
        "fp32_pct_of_peak": 100.0 * achieved / fp32_peak,
        "roofline": {"bound": "alu", "kernel": "walk_kernel (batched far force)", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": None,
                     "peak_source": "148 SMs x 128 FP32 lanes x 2 flop x %.0f MHz (%s sm_max_mhz)"
                                    % (float(peaks.get("sm_max_mhz", 2032.0)), peak_kind)},
        "gpu_launches": None, "clocks": clk,
    }


def _sequential_graph_ms(cl, segn, rows, init, buf, prm0, stream, dev, steps, flush, lists_first=False):
    """The ensemble step one cluster at a time: a context and a captured graph per
    cluster (its own r_out), the 64 graphs launched back to back; step times in ms."""
    import copy

    import torch

    import paper_2110_11658_b300 as p3t
    st = {k: v.clone() for k, v in init.items()}
    per = []
    for k, c in enumerate(cl):
        s0, s1 = int(segn[k]), int(segn[k + 1])
        prm = copy.copy(prm0)
        prm.r_in, prm.r_out, prm.r_list = rows[k][1], rows[k][2], rows[k][3]
        cx = p3t.Context(prm, stream)
        v = {q: st[q][s0:s1] for q in st}
        a = [buf["a"][i][s0:s1] for i in range(3)]
        offs = torch.empty(c.n + 1, dtype=torch.int64, device=dev)
        idx = buf["idx"][16 * s0:16 * s1]
        tot = torch.zeros(1, dtype=torch.int64, device=dev)
        cx.build_tree(v["x"], v["y"], v["z"], v["m"])
        cx.far_force(*a)
        cx.neighbours(offs, idx)  # sizes the row scratch (row mode)
        g = cx.capture_step(v["x"], v["y"], v["z"], v["m"], *a, vx=v["vx"], vy=v["vy"], vz=v["vz"],
                            kick_dt=DT, drift_dt=DT, offsets=offs, idx=idx, total=tot, lists_first=lists_first)
        per.append((cx, g))

    def launch_all():
        for _, g in per:
            g.launch()

    for _ in range(2):
        launch_all()
    res = _dist(_events_ms(stream, launch_all, steps, flush))
    for cx, g in per:
        cx.check()
        g.close()
        cx.close()
    return res


# ---------------------------------------------------------------------------- serving
SERVE_CLUSTERS, SERVE_N_LO, SERVE_N_HI, SERVE_THETA = 256, 1e3, 1e6, 0.5


def serve_run(args):
    """256 device-resident clusters (alternately Plummer and King W0 = 7, Kroupa masses),
    N log-uniform in [1e3, 1e6], theta = 0.5, per-cluster r_out = the paper's r_cut(N).
    A Poisson stream (mean `rate` requests/s, uniform cluster choice, seeded) of distant-
    force-step requests is replayed in real time through (a) the continuous-batching server
    (2 slots), (b) batching on one slot (no overlap), (c) one cluster at a time."""
    import numpy as np
    import torch

    import synth
    from paper_2110_11658_b300.serve import Arena, Server, poisson_arrivals, summary

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t_gen = time.perf_counter()
    sizes = synth.log_uniform_sizes(SERVE_CLUSTERS, SERVE_N_LO, SERVE_N_HI, 20211022)
    cl = [synth.make("plummer" if k % 2 == 0 else "king", int(n), 20211022 + 1 + k, masses="kroupa", w0=7.0)
          for k, n in enumerate(sizes)]
    rows = []
    for c in cl:
        rc = synth.paper_run_params(c.n)["r_cut"]
        rows.append([SERVE_THETA, 0.1 * rc, rc, rc])
    t_gen = time.perf_counter() - t_gen
    warm = poisson_arrivals(args.rate, 200, len(cl), 7)
    big = int(max(sizes))
    cont = dict(n_slots=2, budget=8 * big, max_clusters=256)
    runs = [  # (name, server shape, rate, requests): saturated headline, then lower loads
        ("continuous_2slots", cont, args.rate, args.requests),
        ("batched_1slot", dict(n_slots=1, budget=8 * big, max_clusters=256), args.rate, args.requests),
        ("one_at_a_time", dict(n_slots=1, budget=big, max_clusters=1), args.rate, args.requests),
        ("continuous_2slots_half_rate", cont, args.rate / 2, args.requests // 2),
        ("continuous_2slots_low_rate", cont, 300.0, max(500, args.requests // 5)),
        ("one_at_a_time_low_rate", dict(n_slots=1, budget=big, max_clusters=1), 300.0, max(500, args.requests // 5)),
    ]
    results = {}
    clk = None
    for name, kw, rate, count in runs:
        arr = poisson_arrivals(rate, count, len(cl), 20211022)
        ar = Arena(cl, rows, device=dev)
        srv = Server(ar, dt=DT, **kw)
        srv.run(warm)
        srv.batches = []
        torch.cuda.synchronize(dev)
        clocks = ClockSampler(0) if name == "continuous_2slots" else None
        if clocks:
            clocks.start()
        reqs = srv.run(arr)
        if clocks:
            clk = clocks.stop()
        st = summary(reqs, ar.sizes, srv.batches)
        st.update({"slots": kw["n_slots"], "slot_budget_particles": srv.budget, "rate_per_s": rate,
                   "slot_bytes": srv.bytes_per_slot, "arena_bytes": ar.bytes()})
        results[name] = st
        srv.close()
        del srv, ar
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()
    main_st = results["continuous_2slots"]
    return {
        "metric": "particle far-force evals/sec & interactions/sec at N=1e6 (FP32 % peak); ensemble p50/p99",
        "value": main_st["particles_per_s"], "unit": "particles/s", "n_gpus": 1, "steps": args.requests,
        "warmup": 200, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serve256_poisson%d_n1e3-1e6" % int(args.rate), "n_clusters": len(cl),
                   "resident_particles": int(sum(sizes)), "theta": SERVE_THETA,
                   "r_out": "paper r_cut = 4 tau(N) per cluster", "r_in": "0.1 r_out", "r_list": "r_out",
                   "masses": "Kroupa", "models": "Plummer / King W0 = 7 alternating", "dt": DT,
                   "rate_per_s": args.rate, "requests": args.requests, "generation_s": t_gen},
        "p50_ms": main_st["p50_ms"], "p99_ms": main_st["p99_ms"],
        "serving": results,
        "throughput_vs_one_at_a_time": main_st["particles_per_s"] / results["one_at_a_time"]["particles_per_s"],
        "p99_vs_one_at_a_time": main_st["p99_ms"] / results["one_at_a_time"]["p99_ms"],
        "clocks": clk,
    }


# ---------------------------------------------------------------------------- irregular side
def irregular_run(args):
    """Irregular force and jerk (Eqs. 1, 2) over the neighbour rows of the benchmark
    workload (Plummer 10^6, ~100 neighbours per particle): the mixed and FP64 forms
    timed with CUDA events (L2 flushed between launches), and the oracle over the
    same rows on the host cores."""
    import numpy as np
    import torch

    import oracle
    import paper_2110_11658_b300 as p3t

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    c, w = workload(args.n, 20211022)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d = {k: t(getattr(c, k)) for k in ("x", "y", "z", "m", "vx", "vy", "vz")}
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    out = {}
    offs = torch.empty(c.n + 1, dtype=torch.int64, device=dev)
    idx = None
    for name, prec in (("mixed", p3t.P3T_FP32_MIXED), ("fp64", p3t.P3T_FP64)):
        prm = p3t.Params(theta=w["theta"], r_in=w["r_in"], r_out=w["r_out"], r_list=w["r_list"],
                         leaf_cap=args.leaf_cap, group_size=args.group_size, tile=args.tile, precision=prec)
        ctx = p3t.Context(prm, stream)
        ctx.build_tree(d["x"], d["y"], d["z"], d["m"])
        if idx is None:
            try:
                ctx.neighbours(offs, torch.empty(1, dtype=torch.int32, device=dev))
                total = 0
            except p3t.P3TError as e:
                total = e.total
            idx = torch.empty(max(1, total), dtype=torch.int32, device=dev)
        pairs = ctx.neighbours(offs, idx)
        f = torch.empty(3, c.n, dtype=torch.float64, device=dev)
        jk = torch.empty(3, c.n, dtype=torch.float64, device=dev)
        run = lambda: ctx.irregular(offs, idx, d["x"], d["y"], d["z"], d["m"], d["vx"], d["vy"], d["vz"], f, jk)  # noqa: E731
        for _ in range(max(3, args.warmup)):
            run()
        ts = _events_ms(stream, run, max(3, args.steps), flush)
        ctx.check()
        out[name] = {"ms": float(np.median(ts)), "pairs_per_s": pairs / (float(np.median(ts)) * 1e-3)}
        ctx.close()
    ho, hi = offs.cpu().numpy(), idx[:pairs].cpu().numpy()
    t0 = time.perf_counter()
    oracle.irregular(c.x, c.y, c.z, c.m, c.vx, c.vy, c.vz, w["r_in"], w["r_out"], ho, hi)
    t_cpu = time.perf_counter() - t0
    ms = out["mixed"]["ms"]
    return {
        "metric": "irregular force + jerk over the neighbour rows (Eqs. 1, 2)",
        "value": c.n / (ms * 1e-3), "unit": "particles/s", "n_gpus": 1, "steps": max(3, args.steps),
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 pair arithmetic on f64 differences", "data": "synthetic",
        "config": {"workload": "plummer_kroupa_n%d_nbr100_irregular" % c.n, "n": c.n, "pairs": int(pairs),
                   "r_in": w["r_in"], "r_out": w["r_out"],
                   "l2": "256 MB buffer written between timed launches (L2 is 126 MB)"},
        "forms": out, "fp64_over_mixed": out["fp64"]["ms"] / ms,
        "cpu_baseline": {"value": c.n / t_cpu, "unit": "particles/s", "cores": omp_threads(), "kind": "oracle",
                         "sample": "oracle irregular force and jerk over all %d rows (%d pairs), %.2f s"
                                   % (c.n, int(pairs), t_cpu)},
    }


def core_run(args):
    """Core quantities of the benchmark workload (Plummer 10^6): a seeded random sample
    of min(N, sqrt(5000 N)) particles, their 6 nearest neighbours by brute force over
    all N, and the density-weighted core radius / density / membership.  The oracle's
    search is timed on a subsample and scaled (it is O(sample x N))."""
    import math

    import numpy as np
    import torch

    import oracle
    import paper_2110_11658_b300 as p3t

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    c, w = workload(args.n, 20211022)
    s = int(min(c.n, math.sqrt(5000 * c.n)))
    sample = np.random.default_rng(20211022).choice(c.n, s, replace=False).astype(np.int32)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d = [t(getattr(c, k)) for k in "xyzm"]
    sm = t(sample)
    stream = torch.cuda.current_stream(dev)
    ctx = p3t.Context(p3t.Params(theta=w["theta"], r_in=w["r_in"], r_out=w["r_out"], r_list=w["r_list"]),
                      stream)
    ctx.build_tree(*d)
    res = {}

    def run():
        res["knn"] = ctx.sample_knn6(sm)
        res["core"] = ctx.core_quantities(*d, sm, *res["knn"])

    run()
    brute = ctx.sample_knn6(sm, brute=True)
    same = bool(torch.equal(brute[0], res["knn"][0]) and torch.equal(brute[1], res["knn"][1]))
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    steps = max(3, args.steps)
    ms = float(np.median(_events_ms(stream, lambda: ctx.sample_knn6(sm), steps, flush)))
    ms_brute = float(np.median(_events_ms(stream, lambda: ctx.sample_knn6(sm, brute=True), steps, flush)))
    ctx.check()
    q = res["core"][1]
    sub = sample[:1000]
    t0 = time.perf_counter()
    oracle.knn(c.x, c.y, c.z, sub, 6)
    t_cpu = (time.perf_counter() - t0) * s / len(sub)
    ctx.close()
    return {
        "metric": "6 nearest neighbours of a sqrt(5000 N) sample (core quantities): sampled particles/s",
        "value": s / (ms * 1e-3), "unit": "sampled particles/s", "n_gpus": 1, "steps": steps,
        "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 filter, f64 decisions", "data": "synthetic",
        "config": {"workload": "plummer_kroupa_n%d_core_sample%d" % (c.n, s), "n": c.n, "sample": s,
                   "search": "tree walk (p3t_sample_knn6)",
                   "l2": "256 MB buffer written between timed launches (L2 is 126 MB)"},
        "brute_force": {"ms": ms_brute, "sampled_per_s": s / (ms_brute * 1e-3),
                        "pair_tests_per_s": s * c.n / (ms_brute * 1e-3), "lists_identical": same},
        "core": {"centre": list(map(float, q["centre"])), "r_core": q["r_core"], "rho_core": q["rho_core"],
                 "n_core": q["n_core"]},
        "cpu_baseline": {"value": s / t_cpu, "unit": "sampled particles/s", "cores": omp_threads(),
                         "kind": "oracle", "sample": "oracle brute-force search of 1000 of the %d sampled "
                                                     "particles, scaled to all" % s},
    }


def decomp_run(args):
    """The benchmark workload (Plummer 10^6, theta 0.4, ~100 neighbours) decomposed over
    ranks: under torchrun one rank per GPU (NCCL); otherwise --ranks virtual ranks on one
    GPU, run one after another (what one GPU of a P-GPU run does, without the
    transfers).  Per phase the time of the slowest rank: splitters and partition, range
    build, locally essential trees (export), join, far force, neighbour lists; with the
    bytes each rank receives."""
    import numpy as np
    import torch

    import paper_2110_11658_b300 as p3t
    from paper_2110_11658_b300 import decomp

    rank, local, world = dist_init()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    c, w = workload(args.n, 20211022)
    prm = p3t.Params(theta=w["theta"], r_in=w["r_in"], r_out=w["r_out"], r_list=w["r_list"], leaf_cap=args.leaf_cap,
                     group_size=args.group_size, tile=args.tile, precision=p3t.P3T_FP32_MIXED)
    if world > 1:
        import torch.distributed as dist
        comm = decomp.TorchComm(dist, device=dev)
        mine = [rank]
    else:
        comm = decomp.LocalComm(args.ranks)
        mine = list(range(args.ranks))
    P = comm.size
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731

    def fresh():
        parts = []
        for r in mine:
            sel = np.arange(r, c.n, P)  # an arbitrary first distribution: every P-th particle
            ctx = p3t.Context(prm)
            parts.append(decomp.RankPart(ctx, t(c.x[sel]), t(c.y[sel]), t(c.z[sel]), t(c.m[sel]),
                                         gid=t(sel.astype(np.int64))))
        return parts

    def one_step():
        parts = fresh()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        decomp.decompose(comm, parts, prm)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        far, nbr = [], []
        for p in parts:
            n = p.x.numel()
            a = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3)]
            offs = torch.empty(n + 1, dtype=torch.int64, device=dev)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            p.ctx.far_force(*a)
            e1.record()
            try:  # the list size first (a rank holding the dense core has long rows)
                p.ctx.neighbours(offs, torch.empty(1, dtype=torch.int32, device=dev))
                total = 0
            except p3t.P3TError as err:
                if err.code != p3t.P3T_ERR_CAPACITY:
                    raise
                total = err.total
            idx = torch.empty(max(1, total), dtype=torch.int32, device=dev)
            p.ctx.neighbours(offs, idx)
            e2.record()
            e2.synchronize()
            far.append(e0.elapsed_time(e1))
            nbr.append(e1.elapsed_time(e2))
            p.ctx.check()
        info = [p.info | {"n": p.x.numel()} for p in parts]
        for p in parts:
            p.ctx.close()
        return (t1 - t0) * 1e3, far, nbr, info

    for _ in range(max(1, args.warmup)):
        one_step()
    rows = [one_step() for _ in range(max(1, args.steps))]
    dec_ms = statistics.median(r[0] for r in rows)
    far = [statistics.median(r[1][i] for r in rows) for i in range(len(mine))]
    nbr = [statistics.median(r[2][i] for r in rows) for i in range(len(mine))]
    info = rows[-1][3]
    far_max = dist_max(max(far), world, dev)
    nbr_max = dist_max(max(nbr), world, dev)
    # the same walk on one context holding the whole cluster
    ctx = p3t.Context(prm)
    d = [t(getattr(c, k)) for k in "xyzm"]
    ctx.build_tree(*d)
    a = [torch.empty(c.n, dtype=torch.float32, device=dev) for _ in range(3)]
    ts = []
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.far_force(*a)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ctx.close()
    single_far = statistics.median(ts[1:])
    if rank != 0:
        return None
    per_rank = [{"n": i["n"], "let_nodes_in": i["let_nodes_in"], "let_parts_in": i["let_parts_in"],
                 "let_bytes_in": i["let_nodes_in"] * p3t.P3T_LET_NODE_BYTES + i["let_parts_in"] * p3t.P3T_LET_PART_BYTES,
                 "far_ms": f, "nbr_ms": b} for i, f, b in zip(info, far, nbr)]
    return {
        "metric": "decomposed far-force step: far force per rank (ms) and locally essential tree sizes",
        "value": c.n / (far_max * 1e-3), "unit": "particles/s (far force, slowest rank)", "n_gpus": world,
        "ranks": P, "steps": len(rows), "warmup": args.warmup, "ms_per_step": far_max, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "plummer_kroupa_n%d_theta%.1f_nbr100_ranks%d" % (c.n, THETA, P), "n": c.n,
                   "ranks": P, "ranks_on_gpus": "one per GPU" if world > 1 else "all on one GPU, in turn"},
        "decompose_ms": dec_ms, "far_ms_slowest": far_max, "nbr_ms_slowest": nbr_max,
        "single_context_far_ms": single_far, "bounds": info[0]["bounds"], "top_cells": info[0]["top_cells"],
        "per_rank": per_rank,
    }


def _json_default(o):
    """numpy scalars in result dictionaries."""
    if hasattr(o, "item"):
        return o.item()
    raise TypeError(type(o).__name__)


def main(argv=None):
    args = parse_args(argv)
    if args.workload == "decomp1m":
        line = decomp_run(args)
        if line is not None:
            print(json.dumps(line, default=_json_default))
        return
    if args.workload == "core1m":
        print(json.dumps(core_run(args), default=_json_default))
        return
    if args.workload == "irregular1m":
        print(json.dumps(irregular_run(args), default=_json_default))
        return
    if args.workload == "serve256":
        print(json.dumps(serve_run(args), default=_json_default))
        return
    if args.workload == "king2m":
        king2m_sweep(args)
        return
    if args.workload == "ensemble64":
        print(json.dumps(ensemble_run(args), default=_json_default))
        return
    rank, local, world = dist_init()
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_b300(args, rank, local, world)
    if rank == 0 and line is not None:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
