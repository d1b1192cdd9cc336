"""Autotuner host logic (no GPU): size classes, choice of the fastest
candidate, JSON cache round trip and lookup."""
import pytest

from paper_2103_01216_gb300 import autotune


def test_size_classes_group_by_log2_and_eps():
    assert autotune.size_class(10**9, "u64", 0.25) == autotune.size_class(10**9 + 12345, "u64", 0.26)
    assert autotune.size_class(1 << 20, "u64", 0.5) != autotune.size_class(1 << 22, "u64", 0.5)
    assert autotune.size_class(1 << 20, "u32", 0.5) != autotune.size_class(1 << 20, "u64", 0.5)
    assert autotune.batch_class([256, 4 << 20], "u32", 0.5) == "batch/u32/count2/n2^8-2^22/eps0.50"


def test_pick_best_takes_the_fastest_measurable_candidate():
    cands = [dict(prefix_c=1.0), dict(prefix_c=2.0), dict(prefix_c=4.0)]
    times = {1.0: 9.0, 2.0: None, 4.0: 3.5}
    best, ms, results = autotune.pick_best(cands, lambda c: times[c["prefix_c"]])
    assert best == dict(prefix_c=4.0) and ms == 3.5 and len(results) == 3
    with pytest.raises(RuntimeError):
        autotune.pick_best(cands, lambda c: None)


def test_cache_round_trip_and_lookup(tmp_path, monkeypatch):
    path = str(tmp_path / "t.json")
    monkeypatch.setenv("PIP_TUNE_CACHE", path)
    assert autotune.options_for(1 << 20, "u64", 0.5) == {}
    cache = {autotune.size_class(1 << 20, "u64", 0.5): {"options": {"prefix_c": 2.0, "flags": 64}, "ms": 1.0}}
    autotune.save_cache(cache)
    assert autotune.load_cache() == cache
    assert autotune.options_for((1 << 20) + 7, "u64", 0.5) == {"prefix_c": 2.0, "flags": 64}
    assert autotune.options_for(1 << 24, "u64", 0.5) == {}


def test_candidate_sets_are_valid_options():
    import paper_2103_01216_gb300 as pip

    fields = {f for f, _ in pip.Options._fields_}
    for c in autotune.GRID_CANDIDATES + autotune.CTA_CANDIDATES + autotune.BATCH_CANDIDATES:
        assert set(c) <= fields
