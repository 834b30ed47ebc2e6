"""The batched engine's launch-shape autotuner: seeded sampling and the choice, with a
stand-in for the timed run (no GPU)."""

import pytest

from paper_1603_06757_gb300 import tune


def test_sample_indices_are_distinct_sorted_and_seeded():
    a = tune.sample_indices(1000, 64, 7)
    assert a == sorted(a) and len(set(a)) == 64 and all(0 <= i < 1000 for i in a)
    assert a == tune.sample_indices(1000, 64, 7)
    assert a != tune.sample_indices(1000, 64, 8)
    assert tune.sample_indices(10, 64, 7) == list(range(10))


def test_autotune_picks_the_fastest_shape_and_times_every_candidate():
    calls = []

    def fake(sample, bps, rw):
        calls.append((len(sample), bps, rw))
        return 1.0 + abs(bps - 2) + abs(rw - 8) / 8.0

    codes = [(None, 10 + i) for i in range(500)]
    r = tune.autotune_batch(codes, sample=100, blocks_per_sm=(0, 1, 2, 3), route_work_log10=(7, 8, 9, 10),
                            runner=fake)
    assert (r["blocks_per_sm"], r["route_work_log10"]) == (2, 8)
    assert r["sample"] == 100 and len(r["table"]) == 16
    assert len(calls) == 17 and all(c[0] == 100 for c in calls)  # one warm-up + 16 timed
    assert r["seconds_best"] == 1.0 and r["seconds_worst"] == max(t["seconds"] for t in r["table"])


def test_autotune_needs_codes():
    with pytest.raises(ValueError):
        tune.autotune_batch([], runner=lambda *a: 0.0)
