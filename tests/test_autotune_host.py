"""Host logic of the schedule autotuner: coordinate descent, feasibility of
row_cap, output checks and the JSON cache (no GPU needed)."""
import json

import pytest

from paper_1508_06379_gb300 import autotune


def fake_measure(costs, changed=None):
    """measure() whose stage times are sums of per-option costs."""
    calls = []

    def measure(s):
        calls.append(dict(s))
        search = costs["row_cap"][s["row_cap"]] + costs["search_block"][s["search_block"]]
        lp = (costs["lp_block"][s["lp_block"]] + costs["lp_blocks_per_sm"][s["lp_blocks_per_sm"]] +
              costs["lp_fp64_pivots"][s["lp_fp64_pivots"]])
        ap = costs["apply_block"][s["apply_block"]]
        same = not (changed and changed(s))
        return {"search": search, "lp_small": lp, "apply": ap, "reduce": 1.0}, same

    return measure, calls


COSTS = {
    "row_cap": {16: 0.1, 24: 0.2, 32: 0.3},
    "search_block": {64: 0.3, 128: 0.05, 256: 0.2},
    "lp_block": {32: 0.5, 64: 0.1, 128: 0.2, 192: 0.3, 384: 0.25},
    "lp_blocks_per_sm": {1: 0.2, 2: 0.2, 4: 0.3, 8: 0.2, 16: 0.01, 32: 0.4},
    "apply_block": {64: 0.2, 128: 0.3, 256: 0.1},
    "lp_fp64_pivots": {0: 0.05, 1: 0.5},
}


def test_descent_picks_the_fastest_option_of_every_group():
    measure, calls = fake_measure(COSTS)
    best, report = autotune.descend(measure, k_cap=32, max_count=12)
    assert best == dict(row_cap=16, search_block=128, lp_block=64, lp_blocks_per_sm=16, apply_block=256,
                        lp_fp64_pivots=0)
    # 9 search + 14 + 2 LP + 3 apply candidates, each measured once
    assert len(calls) == 28 and len(report) == 28


def test_row_caps_below_the_widest_row_are_not_tried():
    measure, calls = fake_measure(COSTS)
    best, _ = autotune.descend(measure, k_cap=32, max_count=20)
    assert best["row_cap"] == 24
    assert all(c["row_cap"] >= 20 for c in calls)
    best, _ = autotune.descend(measure, k_cap=16, max_count=10)
    assert best["row_cap"] == 16
    # rows wider than any cap: only k_cap-independent options remain, the default row_cap is kept
    measure, calls = fake_measure(COSTS)
    best, _ = autotune.descend(measure, k_cap=32, max_count=32)
    assert best["row_cap"] == 32 and all(c["row_cap"] == 32 for c in calls)


def test_a_schedule_that_changes_the_output_is_an_error():
    measure, _ = fake_measure(COSTS, changed=lambda s: s["lp_block"] == 32)
    with pytest.raises(RuntimeError):
        autotune.descend(measure, k_cap=32, max_count=12)


def test_buckets_and_keys():
    assert autotune.bucket(1) == 0 and autotune.bucket(1024) == 10 and autotune.bucket(1500) == 11
    assert autotune.bucket(0) == 0
    assert autotune.cache_key("GB300|sm103", 32, 5e5) == "GB300|sm103|k32|n2^19"
    assert autotune.cache_key("GB300|sm103", 32, 5e5, order=2) == "GB300|sm103|k32|o2|n2^19"


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "device_name", lambda: "dev|sm103")
    path = str(tmp_path / "sub" / "schedules.json")
    t = autotune.Autotuner(path)
    assert t.table == {}
    s = dict(autotune.DEFAULT, row_cap=24)
    t.table[autotune.cache_key("dev|sm103", 32, 30000)] = s
    t.save()
    t2 = autotune.Autotuner(path)
    assert t2.lookup(32, 31000) == s and t2.lookup(32, 300000) is None
    assert json.load(open(path)) == t.table
    # an unreadable cache starts empty
    open(path, "w").write("{not json")
    assert autotune.Autotuner(path).table == {}
