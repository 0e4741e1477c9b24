"""Autotuner of the batched executor's launch settings.

Tunes, on a calibration batch, the settings that change speed but never results:
  block_ls   threads per block of the Line-Segment kernel (64, 128, 256);
  warps_px   warps per block of the pT3 / pT5 candidate pre-filters (2, 4, 8);
  persistent Line-Segment kernel: persistent warps pulling the cost-ordered work items from a device
             queue (2), the same list dealt statically (1), or grid-stride over modules (0);
  cap_scale  multiplier of the predicted per-module object capacities: the smallest value whose
             first pass needs no capacity retry on the calibration batch, one step up for margin.
Coordinate descent, each candidate timed as the median of a few CUDA-graph replays. The result is
cached as JSON next to this file, keyed by GPU name and workload class.
"""
from __future__ import annotations

import json
import os
import statistics

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE_DIR = os.path.join(_HERE, "_cache")

SPACE = {"block_ls": [128, 64, 256], "warps_px": [4, 2, 8], "persistent": [2, 1, 0]}
CAP_SCALES = [1.0, 0.75, 0.5, 0.35]


def _time_batch(det, events, stream, reps, **cfg):
    import torch
    from . import lst
    ctx = lst.Context(det, use_graph=1, **cfg)
    ctx.reserve(len(events), max(_nh(e) for e in events), max(_np(e) for e in events))
    ctx.submit(events, stream=stream)
    ctx.sync()
    retries = max(ctx.counts(e)["retries"] for e in range(len(events)))
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.submit(events, stream=stream)
        ctx.sync()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    ctx.close()
    return statistics.median(times), retries


def _nh(e):
    return int(e["x"].shape[0]) if isinstance(e, dict) else e.n_hits


def _np(e):
    return int(e.get("n_pls", 0)) if isinstance(e, dict) else e.n_pls


def tune(det, events, workload="pu200", reps=3, use_cache=True, verbose=False) -> dict:
    """Best settings for this GPU and workload class (a dict of lst_config fields)."""
    import torch
    name = torch.cuda.get_device_name().replace(" ", "_")
    path = os.path.join(CACHE_DIR, f"autotune_{name}_{workload}_b{len(events)}.json")
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)["best"]
        except Exception:
            pass
    stream = torch.cuda.Stream()
    best = {k: v[0] for k, v in SPACE.items()}
    best["cap_scale"] = 1.0
    trials = []
    best_t, _ = _time_batch(det, events, stream, reps, **best)
    trials.append((dict(best), best_t))
    for key, values in SPACE.items():
        for v in values:
            if v == best[key]:
                continue
            cand = dict(best)
            cand[key] = v
            t, retries = _time_batch(det, events, stream, reps, **cand)
            trials.append((cand, t))
            if verbose:
                print("autotune", cand, round(t, 3), "ms")
            if t < best_t and retries == 0:
                best, best_t = cand, t
    # smallest capacity scale that still needs no retry, then one step up
    ok = 1.0
    for sc in CAP_SCALES:
        cand = dict(best, cap_scale=sc)
        t, retries = _time_batch(det, events, stream, 1, **cand)
        trials.append((cand, t))
        if retries:
            break
        ok = sc
    idx = CAP_SCALES.index(ok)
    best["cap_scale"] = CAP_SCALES[max(0, idx - 1)]
    result = {"best": best, "best_ms": best_t, "trials": [{"cfg": c, "ms": t} for c, t in trials]}
    try:
        os.makedirs(CACHE_DIR, exist_ok=True)
        with open(path, "w") as f:
            json.dump(result, f, indent=1)
    except OSError:
        pass
    return best
