"""Autotuner search logic on a synthetic cost function (no GPU)."""
import json

import pytest

from paper_2110_11658_b300 import autotune


def _cost(cfg):
    # a separable cost with its minimum at G = 64 on two warps, tile = 128, leaf_cap = 8,
    # lists after the far force
    return (abs(cfg["group_size"] - 64) / 32 + abs(cfg["tile"] - 128) / 64 + abs(cfg["leaf_cap"] - 8) / 8
            + (0.0 if cfg["threads_per_group"] == 64 else 0.5) + 0.25 * cfg["lists_first"] + 1.0)


def test_tuner_finds_minimum_in_three_stages():
    calls = []
    tuner = autotune.Tuner(lambda c: calls.append(c) or _cost(c), repeats=1)
    res = tuner.tune()
    assert res.best == {"group_size": 64, "threads_per_group": 64, "tile": 128, "leaf_cap": 8, "lists_first": 0}
    assert res.best_ms == pytest.approx(1.0)
    # stage 1: (G, threads) in (32, 32), (64, 32), (64, 64), (128, 32), (128, 128) x 4 tiles
    # at leaf_cap 16; stage 2: the two other leaf capacities; stage 3: the other order
    assert len(calls) == 20 + 2 + 1
    assert all(c["leaf_cap"] == 16 and c["lists_first"] == 0 for c in calls[:20])
    assert {(c["group_size"], c["threads_per_group"]) for c in calls[:20]} == {
        (32, 32), (64, 32), (64, 64), (128, 32), (128, 128)}
    assert {c["leaf_cap"] for c in calls[20:22]} == {8, 32}
    assert calls[22] == dict(res.best, lists_first=1)


def test_tuner_picks_lists_first_when_faster():
    res = autotune.Tuner(lambda c: _cost(c) - 0.5 * c["lists_first"], repeats=1).tune()
    assert res.best["lists_first"] == 1 and res.best["group_size"] == 64


def test_threads_per_group_validity():
    ok = {"group_size": 64, "threads_per_group": 64, "tile": 64, "leaf_cap": 16}
    assert autotune.valid(ok)
    assert not autotune.valid(dict(ok, threads_per_group=96))
    assert not autotune.valid(dict(ok, group_size=128))  # more targets than threads
    assert autotune.valid(dict(ok, group_size=128, threads_per_group=32))  # 4 per lane


def test_tuner_takes_median_of_repeats():
    seq = iter([5.0, 1.0, 3.0] + [9.0] * 100)
    tuner = autotune.Tuner(lambda c: next(seq), repeats=3, group_sizes=(32,), tiles=(64,), leaf_caps=(16,),
                           orders=(0,))
    res = tuner.tune()
    assert res.best_ms == 3.0 and len(res.table) == 1


def test_tuner_skips_invalid_shapes():
    seen = []
    tuner = autotune.Tuner(lambda c: seen.append(c) or 1.0, repeats=1, group_sizes=(32, 256),
                           tiles=(64, 512), leaf_caps=(16,))
    tuner.tune()
    assert seen == [{"group_size": 32, "threads_per_group": 32, "tile": 64, "leaf_cap": 16, "lists_first": 0},
                    {"group_size": 32, "threads_per_group": 32, "tile": 64, "leaf_cap": 16, "lists_first": 1}]
    with pytest.raises(ValueError):
        autotune.Tuner(lambda c: 1.0, group_sizes=(256,), tiles=(64,)).tune()


def test_tuner_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    key = autotune.workload_key("B300", [10000, 20000], 0, 0.4)
    res = autotune.Tuner(_cost, repeats=1, cache_path=path).tune(key)
    assert not res.cached
    data = json.load(open(path))
    assert data[key]["best"] == res.best

    def boom(cfg):
        raise AssertionError("a cached workload must not be re-timed")

    again = autotune.Tuner(boom, cache_path=path).tune(key)
    assert again.cached and again.best == res.best and again.best_ms == res.best_ms
    other = autotune.workload_key("B300", [10000, 20001], 0, 0.4)
    assert other != key
    assert autotune.workload_key("B300", [10000, 20000], 0, 0.4) == key
