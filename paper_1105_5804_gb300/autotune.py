"""Autotuner for batched Swendsen-Wang chains.

Picks, for a batch of chains, the labeling tile shape and how one sweep is
scheduled.  Tile shapes: 32 rows by 256, 128 or 64 columns (the library is
built once per width); a lattice whose side is not a multiple of the width
leaves a ragged last tile column whose threads idle, so small and odd-sized
chains favour narrow tiles and large ones wide tiles (fewer seams to merge).
Schedules: one launch per step over all tiles (SW_BATCH_PHASES), or one
persistent cooperative launch per sweep with a chosen number of CTAs per SM
(SW_BATCH_PERSISTENT; the merge runs between grid barriers).  Every
candidate is timed with CUDA events on a clone of the batch (same sizes,
couplings and state counts, other seeds), so the chains being tuned for are
not advanced.  Results are cached in a JSON file keyed by the GPU name and
the batch's shape (sizes, q, number of chains).
"""
import hashlib
import json
import os

from . import _lib as sw

CACHE = os.environ.get("SWCCL_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "swccl", "autotune.json"))


def _signature(L, q):
    h = hashlib.sha1()
    h.update(",".join("%d:%d" % (a, b) for a, b in sorted(zip(L, q))).encode())
    return "%d-%s" % (len(L), h.hexdigest()[:16])


def _gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(db):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + ".tmp.%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def time_batch(b, sweeps):
    """Milliseconds for `sweeps` sweeps of batch b (CUDA events on its stream)."""
    import torch
    st = torch.cuda.ExternalStream(sw.sw_batch_stream(b))
    sw.sw_batch_sync(b)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    sw.sw_batch_sweep(b, sweeps)
    e1.record(st)
    sw.sw_batch_sync(b)
    return e0.elapsed_time(e1)


def candidates(max_blocks_per_sm=4):
    """Schedules tried for each tile width."""
    out = [{"schedule": sw.SW_BATCH_PHASES, "blocks_per_sm": 0}]
    for k in range(1, max_blocks_per_sm + 1):
        out.append({"schedule": sw.SW_BATCH_PERSISTENT, "blocks_per_sm": k})
    return out


def tune(L, q, beta, convention=sw.SW_CONV_AUTO, sweeps=3, use_cache=True, max_blocks_per_sm=4,
         tile_widths=sw.TILE_WIDTHS):
    """Best tile width and schedule for chains (L, q, beta): a dict with
    tile_w, schedule, blocks_per_sm, ms_per_sweep and all timings."""
    key = "%s|%s|%s" % (_gpu_name(), _signature(L, q), ",".join(str(w) for w in tile_widths))
    db = _load() if use_cache else {}
    if use_cache and key in db:
        return dict(db[key], cached=True)
    timings = []
    for tw in tile_widths:
        clone = sw.sw_batch_create(L, q, beta, [0x5EED + r for r in range(len(L))], convention, True, tile_w=tw)
        try:
            sw.sw_batch_sweep(clone, 1)                       # warm-up and graph capture
            for c in candidates(max_blocks_per_sm):
                sw.sw_batch_set_schedule(clone, c["schedule"], c["blocks_per_sm"])
                sw.sw_batch_sweep(clone, 1)
                ms = time_batch(clone, sweeps) / sweeps
                timings.append(dict(c, tile_w=tw, ms_per_sweep=ms))
        finally:
            sw.sw_batch_destroy(clone)
    best = min(timings, key=lambda t: t["ms_per_sweep"])
    res = {"tile_w": best["tile_w"], "schedule": best["schedule"], "blocks_per_sm": best["blocks_per_sm"],
           "ms_per_sweep": best["ms_per_sweep"], "timings": timings}
    if use_cache:
        db[key] = res
        _store(db)
    return dict(res, cached=False)


def create_tuned(L, q, beta, seed, convention=sw.SW_CONV_AUTO, hot_start=False, stream=0, **tune_kw):
    """A batch of these chains built with the tuned tile width and schedule;
    returns (batch, choice)."""
    choice = tune(L, q, beta, convention, **tune_kw)
    b = sw.sw_batch_create(L, q, beta, seed, convention, hot_start, stream, tile_w=choice["tile_w"])
    apply(b, choice)
    return b, choice


def apply(b, choice):
    sw.sw_batch_set_schedule(b, choice["schedule"], choice["blocks_per_sm"])
