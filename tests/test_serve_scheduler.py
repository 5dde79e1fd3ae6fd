"""Serving policy (admission by footprint, continuous batching) on the CPU."""
import heapq

import numpy as np
import pytest

from paper_2110_11658_b300.serve import Request, Scheduler, latency_stats, poisson_arrivals


def test_batch_respects_budget_and_arrival_order():
    sizes = [40, 30, 50, 10, 20]
    s = Scheduler(sizes, n_slots=2, budget=100)
    for i, k in enumerate([0, 1, 2, 3, 4]):
        s.submit(Request(i, k, float(i)))
    b = s.form_batch()
    # 40 + 30 fit, 50 does not: the batch stops there (no overtaking by 10 or 20)
    assert [r.cluster for r in b.requests] == [0, 1] and b.particles == 70
    b2 = s.form_batch()
    assert [r.cluster for r in b2.requests] == [2, 3, 4] and b2.particles == 80
    assert s.form_batch() is None  # both slots busy: backpressure
    s.complete(b.bid)
    assert s.free_slots == [b.slot]


def test_same_cluster_steps_stay_in_order():
    s = Scheduler([10, 10, 10], n_slots=3, budget=100)
    for i, k in enumerate([0, 0, 1, 0]):
        s.submit(Request(i, k, float(i)))
    b1 = s.form_batch()
    assert [r.rid for r in b1.requests] == [0, 2]  # one step of cluster 0 per batch
    b2 = s.form_batch()
    assert b2 is None  # cluster 0 is in flight, its later steps wait
    s.complete(b1.bid)
    b3 = s.form_batch()
    assert [r.rid for r in b3.requests] == [1]
    s.complete(b3.bid)
    b4 = s.form_batch()
    assert [r.rid for r in b4.requests] == [3]


def test_refuses_cluster_larger_than_budget_and_caps_segments():
    s = Scheduler([5, 500], n_slots=1, budget=100, max_clusters=2)
    with pytest.raises(ValueError):
        s.submit(Request(0, 1, 0.0))
    s2 = Scheduler([1] * 5, n_slots=1, budget=100, max_clusters=2)
    for i in range(5):
        s2.submit(Request(i, i, 0.0))
    assert len(s2.form_batch().requests) == 2


def _simulate(sizes, arrivals, n_slots, budget, cost_per_particle=1e-6, launch_cost=1e-4):
    """Event-driven run of the policy: a batch of P particles takes
    launch_cost + P * cost_per_particle seconds on its slot."""
    s = Scheduler(sizes, n_slots, budget)
    reqs = [Request(i, c, t) for i, (t, c) in enumerate(arrivals)]
    events, t, nxt, done = [], 0.0, 0, 0
    batches = []
    while done < len(reqs):
        while nxt < len(reqs) and reqs[nxt].t_arrival <= t:
            s.submit(reqs[nxt])
            nxt += 1
        while True:
            b = s.form_batch()
            if b is None:
                break
            for r in b.requests:
                r.t_launch = t
            batches.append(b)
            heapq.heappush(events, (t + launch_cost + b.particles * cost_per_particle, b.bid))
        t_next_arr = reqs[nxt].t_arrival if nxt < len(reqs) else np.inf
        if events and events[0][0] <= t_next_arr:
            t, bid = heapq.heappop(events)
            for r in s.complete(bid).requests:
                r.t_done = t
                done += 1
        else:
            t = t_next_arr
    return reqs, batches


def test_simulated_stream_completes_with_invariants():
    rng = np.random.default_rng(3)
    sizes = list(rng.integers(1000, 100000, 32))
    arr = poisson_arrivals(500.0, 2000, 32, 7)
    reqs, batches = _simulate(sizes, arr, n_slots=2, budget=400000)
    assert all(b.particles <= 400000 for b in batches)
    assert all(np.isfinite(r.t_done) and r.t_done >= r.t_launch >= r.t_arrival for r in reqs)
    # per-cluster steps complete in arrival order, never overlapping
    by = {}
    for r in sorted(reqs, key=lambda r: r.rid):
        if r.cluster in by:
            assert r.t_launch >= by[r.cluster].t_done
        by[r.cluster] = r
    st = latency_stats(reqs)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    # batching more than one slot's worth of requests at a time pays: fewer batches than requests
    assert len(batches) < len(reqs)


def test_continuous_batching_beats_one_at_a_time_under_load():
    rng = np.random.default_rng(4)
    sizes = list(rng.integers(1000, 100000, 32))
    arr = poisson_arrivals(2000.0, 1500, 32, 8)
    r_batch, _ = _simulate(sizes, arr, n_slots=2, budget=800000, launch_cost=2e-3)
    r_one, _ = _simulate(sizes, arr, n_slots=1, budget=max(sizes), launch_cost=2e-3)
    assert latency_stats(r_batch)["p99_ms"] < latency_stats(r_one)["p99_ms"]


def test_poisson_arrivals_statistics():
    arr = poisson_arrivals(2000.0, 20000, 256, 11)
    t = np.array([a[0] for a in arr])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert abs(np.diff(t).mean() * 2000.0 - 1.0) < 0.03
    cl = np.array([a[1] for a in arr])
    assert cl.min() >= 0 and cl.max() < 256 and len(np.unique(cl)) == 256
