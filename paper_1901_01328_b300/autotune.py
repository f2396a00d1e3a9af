"""Autotuner for the library's tuning knobs: measures the candidates on the
current GPU and sets the knobs (sbh_set_knob) to the fastest.

  sort path    below some size one onesweep kernel per pass (decoupled
               look-back over tiles) beats the per-chunk count / scan /
               scatter passes, whose extra launches and count read only pay
               off on large sorts.  The tuner times both at sizes around the
               crossover and sets SBH_KNOB_SORT_CHUNKED_MIN to the smallest
               size from which the chunked passes win.
  merge cuts   small merges let each CTA search its own cuts; large ones
               search them in a separate parallel kernel first.  The tuner
               times both and sets SBH_KNOB_MERGE_SEARCH_MIN_TILES.
  scatter      the chunked scatter's tile and CTA shape (4096 rows x 512
               threads, 2048 x 256, 8192 x 1024: more rows per tile mean
               fewer tiles and barriers, fewer mean more CTAs per SM to hide
               latency).  The tuner times the plain sort with each on large
               sorts and sets SBH_KNOB_SCATTER_GEOM to the fastest.
  digit width  stays 8 bits: a digit's per-warp counters, packed two per
               word, and its 256-entry scans fit the two-CTA shared-memory
               budget of the scatter; 11-bit digits (2048 counters per warp)
               would not, and would save passes only on keys of more than
               about 40 significant bits.
  schedule     for many small windows, `batched_schedule` times the batched
               (composite-key) and per-window schedules of
               pipeline.batched_windows on a sample and returns the faster.

Results can be saved to and loaded from a JSON file, keyed by device name.
All timing is by CUDA events on the current stream (median of repeats).
"""
from __future__ import annotations

import json
import os
import statistics

import torch

from . import sbh


def _time(fn, reps=5, warm=2):
    ts = []
    for r in range(reps + warm):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        if r >= warm:
            ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def _keys(n, seed):
    import gen
    return torch.from_numpy(gen.mixed_keys(n, seed=seed)).cuda()


def tune_sort_threshold(sizes=(1 << 19, 1 << 20, 3 << 19, 1 << 21, 3 << 20, 1 << 22), seed=11):
    """Times the sort of mixed 64-bit keys with each path at each size; sets
    and returns the chosen threshold with the timings (ms)."""
    old = sbh.get_knob(sbh.KNOB_SORT_CHUNKED_MIN)
    timings = {}
    try:
        for n in sizes:
            keys, ptrs = sbh.extract(_keys(n, seed), 0, n)
            out = (torch.empty_like(keys), torch.empty_like(ptrs))
            row = {}
            for path, thr in (("onesweep", 1 << 40), ("chunked", 0)):
                sbh.set_knob(sbh.KNOB_SORT_CHUNKED_MIN, thr)
                scr = torch.empty(sbh.sort_scratch_bytes(n), dtype=torch.uint8, device="cuda")
                row[path] = _time(lambda: sbh.sbh_kpa_sort(keys, ptrs, out[0], out[1], scratch=scr))
            timings[n] = row
    finally:
        sbh.set_knob(sbh.KNOB_SORT_CHUNKED_MIN, old)
    wins = [n for n in sizes if timings[n]["chunked"] < timings[n]["onesweep"]]
    # the smallest size from which the chunked passes keep winning
    choice = sizes[-1] * 2
    for n in reversed(sizes):
        if n in wins:
            choice = n
        else:
            break
    sbh.set_knob(sbh.KNOB_SORT_CHUNKED_MIN, choice)
    return {"knob": "SBH_KNOB_SORT_CHUNKED_MIN", "value": choice, "timings_ms": timings}


def tune_merge_search(totals=(1 << 20, 1 << 21, 1 << 22, 1 << 23), seed=12):
    """Times two-run merges with the cuts searched per CTA and by the separate
    kernel; sets and returns the tile-count threshold."""
    old = sbh.get_knob(sbh.KNOB_MERGE_SEARCH_MIN_TILES)
    timings = {}
    try:
        for total in totals:
            col = _keys(total, seed)
            a = sbh.sort(*sbh.extract(col, 0, total // 2))
            b = sbh.sort(*sbh.extract(col, total // 2, total - total // 2))
            ok = torch.empty(total, dtype=torch.uint64, device="cuda")
            op = torch.empty(total, dtype=torch.uint32, device="cuda")
            row = {}
            for path, thr in (("per_cta", 1 << 40), ("separate", 0)):
                sbh.set_knob(sbh.KNOB_MERGE_SEARCH_MIN_TILES, thr)
                row[path] = _time(lambda: sbh.sbh_kpa_merge([a, b], ok, op))
            timings[total] = row
    finally:
        sbh.set_knob(sbh.KNOB_MERGE_SEARCH_MIN_TILES, old)
    tiles = {t: (t + 2047) // 2048 for t in totals}
    choice = tiles[totals[-1]] * 2
    for t in reversed(totals):
        if timings[t]["separate"] < timings[t]["per_cta"]:
            choice = tiles[t] - 1
        else:
            break
    sbh.set_knob(sbh.KNOB_MERGE_SEARCH_MIN_TILES, choice)
    return {"knob": "SBH_KNOB_MERGE_SEARCH_MIN_TILES", "value": choice, "timings_ms": timings}


def tune_scatter_geometry(sizes=(1 << 25, 1 << 26), seed=13):
    """Times the plain sort of mixed 64-bit keys (chunked passes) with each
    scatter geometry; sets and returns the fastest over the sizes."""
    old = sbh.get_knob(sbh.KNOB_SCATTER_GEOM)
    timings = {}
    try:
        for n in sizes:
            keys, ptrs = sbh.extract(_keys(n, seed), 0, n)
            out = (torch.empty_like(keys), torch.empty_like(ptrs))
            scr = torch.empty(sbh.sort_scratch_bytes(n), dtype=torch.uint8, device="cuda")
            row = {}
            for geom in sorted(sbh.SCATTER_GEOMS):
                sbh.set_knob(sbh.KNOB_SCATTER_GEOM, geom)
                row[geom] = _time(lambda: sbh.sbh_kpa_sort(keys, ptrs, out[0], out[1], scratch=scr))
            timings[n] = row
            del keys, ptrs, out, scr
    finally:
        sbh.set_knob(sbh.KNOB_SCATTER_GEOM, old)
    total = {g: sum(timings[n][g] for n in sizes) for g in sbh.SCATTER_GEOMS}
    choice = min(total, key=total.get)
    sbh.set_knob(sbh.KNOB_SCATTER_GEOM, choice)
    return {"knob": "SBH_KNOB_SCATTER_GEOM", "value": choice, "geometry": sbh.SCATTER_GEOMS[choice],
            "timings_ms": timings}


def batched_schedule(key_col, val_col, offsets, K=3, sample_windows=64):
    """Times both schedules of pipeline.batched_windows on the first
    sample_windows windows and returns ("batched" | "loop", timings)."""
    import time

    import numpy as np

    from . import pipeline

    off = np.asarray(offsets, dtype=np.uint64)[: sample_windows + 1]
    t = {}
    for sched in ("batched", "loop"):
        pipeline.batched_windows(key_col, val_col, off, K=K, schedule=sched)  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pipeline.batched_windows(key_col, val_col, off, K=K, schedule=sched)
        torch.cuda.synchronize()
        t[sched] = 1e3 * (time.perf_counter() - t0)
    return min(t, key=t.get), t


def autotune(cache=None, quick=False):
    """Tunes every knob (or loads them from `cache`, a JSON file, when it
    holds this device's values); returns the chosen values.  quick: smaller
    sorts for the scatter geometry."""
    dev = torch.cuda.get_device_name()
    if cache and os.path.exists(cache):
        with open(cache) as f:
            saved = json.load(f).get(dev)
        if saved and "SBH_KNOB_SCATTER_GEOM" in saved:
            sbh.set_knob(sbh.KNOB_SORT_CHUNKED_MIN, saved["SBH_KNOB_SORT_CHUNKED_MIN"])
            sbh.set_knob(sbh.KNOB_MERGE_SEARCH_MIN_TILES, saved["SBH_KNOB_MERGE_SEARCH_MIN_TILES"])
            sbh.set_knob(sbh.KNOB_SCATTER_GEOM, saved["SBH_KNOB_SCATTER_GEOM"])
            return saved
    res = {"SBH_KNOB_SORT_CHUNKED_MIN": tune_sort_threshold()["value"],
           "SBH_KNOB_MERGE_SEARCH_MIN_TILES": tune_merge_search()["value"],
           "SBH_KNOB_SCATTER_GEOM": tune_scatter_geometry(sizes=(1 << 24,) if quick else (1 << 25, 1 << 26))["value"]}
    if cache:
        data = {}
        if os.path.exists(cache):
            with open(cache) as f:
                data = json.load(f)
        data[dev] = res
        with open(cache, "w") as f:
            json.dump(data, f, indent=1)
    return res
