"""Host logic of the batch autotuner on the CPU: the fastest candidate over
tile widths and schedules is chosen, results are cached per GPU name and
batch shape (the order of the chains does not matter), and a cached choice
is reused without timing.  The device calls are stubs here; the GPU tests
tune real batches."""
import json

import pytest

from paper_1105_5804_gb300 import autotune


@pytest.fixture
def stubbed(monkeypatch, tmp_path):
    calls = {"created": 0, "schedule": None, "timed": [], "widths": []}
    ms_of = {}
    for tw, scale in ((256, 1.0), (128, 1.2), (64, 0.9)):
        ms_of[(tw, autotune.sw.SW_BATCH_PHASES, 0)] = 3.0 * scale
        for k, ms in zip(range(1, 5), (5.0, 2.5, 1.5, 1.75)):
            ms_of[(tw, autotune.sw.SW_BATCH_PERSISTENT, k)] = ms * scale

    def create(L, q, beta, seeds, conv, hot, tile_w=256):
        calls["created"] += 1
        calls["widths"].append(tile_w)
        return tile_w

    def set_schedule(b, schedule, bps):
        calls["schedule"] = (b, schedule, bps)

    def time_batch(b, sweeps):
        calls["timed"].append(calls["schedule"])
        return ms_of[calls["schedule"]] * sweeps

    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "GPU-A")
    monkeypatch.setattr(autotune.sw, "sw_batch_create", create)
    monkeypatch.setattr(autotune.sw, "sw_batch_sweep", lambda b, n: None)
    monkeypatch.setattr(autotune.sw, "sw_batch_set_schedule", set_schedule)
    monkeypatch.setattr(autotune.sw, "sw_batch_destroy", lambda b: None)
    monkeypatch.setattr(autotune, "time_batch", time_batch)
    return calls, tmp_path / "tune.json"


def test_fastest_candidate_is_chosen_and_cached(stubbed):
    calls, cache = stubbed
    r = autotune.tune([64, 128, 256], [2, 2, 3], [0.4, 0.44, 0.5])
    assert (r["tile_w"], r["schedule"], r["blocks_per_sm"]) == (64, autotune.sw.SW_BATCH_PERSISTENT, 3)
    assert abs(r["ms_per_sweep"] - 1.5 * 0.9) < 1e-12 and not r["cached"]
    assert sorted(calls["widths"]) == [64, 128, 256]          # one clone per tile width
    assert len(r["timings"]) == 3 * len(autotune.candidates()) == len(calls["timed"])
    db = json.loads(cache.read_text())
    assert len(db) == 1 and next(iter(db)).startswith("GPU-A|3-")


def test_cached_choice_is_reused_for_the_same_shape_in_any_order(stubbed):
    calls, _ = stubbed
    autotune.tune([64, 128, 256], [2, 2, 3], [0.4, 0.44, 0.5])
    n = len(calls["timed"])
    r = autotune.tune([256, 64, 128], [3, 2, 2], [0.5, 0.4, 0.44])
    assert r["cached"] and len(calls["timed"]) == n and calls["created"] == 3
    autotune.tune([64, 128, 256], [2, 2, 2], [0.4, 0.44, 0.5])      # other q: another shape
    assert calls["created"] == 6


def test_other_gpu_or_no_cache_times_again(stubbed, monkeypatch):
    calls, _ = stubbed
    autotune.tune([64, 64], [2, 2], [0.4, 0.4])
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "GPU-B")
    autotune.tune([64, 64], [2, 2], [0.4, 0.4])
    assert calls["created"] == 6
    r = autotune.tune([64, 64], [2, 2], [0.4, 0.4], use_cache=False)
    assert calls["created"] == 9 and not r["cached"]
