"""Host logic of the batch autotuner: tune keys and the JSON cache file
(st_tune_key / st_tune_load / st_tune_store; no GPU needed)."""
import json

import pytest


def test_tune_key_buckets_by_log2_prims_resolution_and_mode(stlib):
    assert stlib.st_tune_key(1024, 1920, 1080, 0) == "m0_n10_1920x1080"
    assert stlib.st_tune_key(1400, 1920, 1080, 1) == "m1_n10_1920x1080"   # log2 1400 = 10.45
    assert stlib.st_tune_key(1500, 256, 256, 2) == "m2_n11_256x256"       # log2 1500 = 10.55
    assert stlib.st_tune_key(1, 8, 8, 0) == "m0_n0_8x8"
    with pytest.raises(stlib.StError):
        stlib.st_tune_key(0, 256, 256, 0)


def test_cache_round_trip_and_replace(stlib, tmp_path):
    p = tmp_path / "tune.json"
    assert stlib.st_tune_load(p, "m0_n10_1920x1080") is None          # no file yet
    stlib.st_tune_store(p, "m0_n10_1920x1080", stlib.st_tune(16, 24, 0.05, 1.5))
    stlib.st_tune_store(p, "m1_n5_256x256", stlib.st_tune(8, 12, 0.15, 0.25))
    stlib.st_tune_store(p, "m0_n10_1920x1080", stlib.st_tune(32, 32, 0.15, 1.25))   # replace
    d = json.loads(p.read_text())                                     # valid JSON for other tools
    assert d["st_autotune"] == 1 and set(d["entries"]) == {"m0_n10_1920x1080", "m1_n5_256x256"}
    t = stlib.st_tune_load(p, "m0_n10_1920x1080")
    assert (t.tile, t.max_new_per_turn) == (32, 32) and abs(t.depth_slab_frac - 0.15) < 1e-7
    t = stlib.st_tune_load(p, "m1_n5_256x256")
    assert (t.tile, t.max_new_per_turn, t.ms) == (8, 12, 0.25)
    assert stlib.st_tune_load(p, "m0_n9_1920x1080") is None           # absent key


def test_cache_written_by_hand_with_extra_fields(stlib, tmp_path):
    p = tmp_path / "tune.json"
    p.write_text(json.dumps({"comment": "hand made", "st_autotune": 1, "entries": {
        "m0_n6_256x256": {"tile": 8, "max_new_per_turn": 6, "depth_slab_frac": 0.5, "note": [1, {"a": None}]}}}))
    t = stlib.st_tune_load(p, "m0_n6_256x256")
    assert (t.tile, t.max_new_per_turn) == (8, 6) and t.depth_slab_frac == 0.5 and t.ms == 0.0


def test_invalid_entries_and_files_are_rejected(stlib, tmp_path):
    p = tmp_path / "tune.json"
    for bad in (stlib.st_tune(12, 24, 0.05, 0), stlib.st_tune(16, 0, 0.05, 0), stlib.st_tune(16, 1025, 0.05, 0),
                stlib.st_tune(16, 24, 0.0, 0)):
        with pytest.raises(stlib.StError):
            stlib.st_tune_store(p, "k", bad)
    with pytest.raises(stlib.StError):
        stlib.st_tune_store(p, 'bad"key', stlib.st_tune(16, 24, 0.05, 0))
    # a malformed existing file is neither read nor overwritten
    p.write_text('{"st_autotune": 1, "entries": {"k": {"tile": 16,')
    assert stlib.st_tune_load(p, "k") is None
    with pytest.raises(stlib.StError):
        stlib.st_tune_store(p, "k2", stlib.st_tune(16, 24, 0.05, 0))
    assert p.read_text().endswith('"tile": 16,')
    # an entry with an unusable tile size is treated as absent
    p.write_text(json.dumps({"entries": {"k": {"tile": 12, "max_new_per_turn": 24, "depth_slab_frac": 0.05}}}))
    assert stlib.st_tune_load(p, "k") is None
