"""Autotuner search logic on a synthetic cost function (no GPU)."""
import json

import pytest

from paper_2110_11658_b300 import autotune


def _cost(cfg):
    # a separable cost with its minimum at G = 64, tile = 128, leaf_cap = 8
    return abs(cfg["group_size"] - 64) / 32 + abs(cfg["tile"] - 128) / 64 + abs(cfg["leaf_cap"] - 8) / 8 + 1.0


def test_tuner_finds_minimum_in_two_stages():
    calls = []
    tuner = autotune.Tuner(lambda c: calls.append(c) or _cost(c), repeats=1)
    res = tuner.tune()
    assert res.best == {"group_size": 64, "tile": 128, "leaf_cap": 8}
    assert res.best_ms == pytest.approx(1.0)
    # stage 1: 3 x 4 shapes at leaf_cap 16; stage 2: the two other leaf capacities
    assert len(calls) == 12 + 2
    assert all(c["leaf_cap"] == 16 for c in calls[:12])
    assert {c["leaf_cap"] for c in calls[12:]} == {8, 32}


def test_tuner_takes_median_of_repeats():
    seq = iter([5.0, 1.0, 3.0] + [9.0] * 100)
    tuner = autotune.Tuner(lambda c: next(seq), repeats=3, group_sizes=(32,), tiles=(64,), leaf_caps=(16,))
    res = tuner.tune()
    assert res.best_ms == 3.0 and len(res.table) == 1


def test_tuner_skips_invalid_shapes():
    seen = []
    tuner = autotune.Tuner(lambda c: seen.append(c) or 1.0, repeats=1, group_sizes=(32, 256),
                           tiles=(64, 512), leaf_caps=(16,))
    tuner.tune()
    assert seen == [{"group_size": 32, "tile": 64, "leaf_cap": 16}]
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
