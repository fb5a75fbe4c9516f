"""Autotuner for the launch shapes of the tracking and refit kernels (tpc_tuning).

For every tunable kernel in turn (coordinate descent, the others held at their current best) the
tuner sweeps threads per CTA, CTAs per SM and, for the following, the number of chains taken per
queue grab, and times the kernel's stage with the per-stage CUDA events of the library
(tpc_profile_*), median of `reps` calls, on the caller's workload.  Launch shapes never change
results, so the search is free to pick any candidate.  The result is kept in a JSON cache keyed
by GPU name, SM count and a workload signature (events, clusters per event bucket).
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import numpy as np
import torch

from . import capi

KERNELS = ["grid", "links", "chains", "follow", "select", "merge", "refit", "refit_grad"]
# candidate (block, ctas_per_sm, chunk) per kernel; 0 = library default
CANDIDATES = {
    "grid": dict(block=[64, 128, 256], ctas=[0, 8, 16, 32], chunk=[0]),
    "links": dict(block=[64, 96, 128], ctas=[4, 6, 8, 10, 16], chunk=[0, 1, 2]),   # 0: slab order, 1: rows staged in smem, 2: cluster order
    "chains": dict(block=[64, 128, 256], ctas=[0, 8, 16, 32], chunk=[0]),
    "follow": dict(block=[64, 96, 128], ctas=[4, 8, 12, 16], chunk=[1, 2, 4]),
    "select": dict(block=[256, 512, 1024], ctas=[1, 2, 4], chunk=[0]),
    "merge": dict(block=[64, 128, 256, 512], ctas=[4, 8, 16], chunk=[0]),
    "refit": dict(block=[64, 128], ctas=[2, 4, 8, 16], chunk=[0]),
    "refit_grad": dict(block=[64, 128], ctas=[2, 4, 8], chunk=[0, 1]),  # 0: checkpoints, 1: stored states
}
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_cache.json")


def workload_key(n_events, n_clusters):
    per_event = max(n_clusters, 1) / max(n_events, 1)
    dev = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s|sm%d|ev%d|cl2^%d" % (dev.name, dev.multi_processor_count, n_events, int(round(math.log2(per_event))))


def to_struct(d):
    t = capi.tpc_tuning()
    for k, name in enumerate(KERNELS):
        b, c, h = d.get(name, (0, 0, 0))
        t.block[k], t.ctas_per_sm[k], t.chunk[k] = int(b), int(c), int(h)
    return t


def load(key, path=CACHE):
    if not os.path.exists(path):
        return None
    return json.load(open(path)).get(key)


def store(key, entry, path=CACHE):
    data = json.load(open(path)) if os.path.exists(path) else {}
    data[key] = entry
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _stage_times(ctx, run, reps):
    """Median per-stage milliseconds of `reps` calls of run()."""
    per = []
    for _ in range(reps):
        ctx.tpc_profile_read(reset=True)
        run()
        torch.cuda.synchronize()
        ms, n = ctx.tpc_profile_read(reset=True)
        per.append(ms)
    return {k: float(np.median([p.get(k, 0.0) for p in per])) for k in per[0]}


def autotune(ctx, run, reps=3, candidates=CANDIDATES, log=None):
    """Coordinate descent over the kernels of CANDIDATES.  run() must perform one call of the
    path (e.g. tpc_track_batch + tpc_refit_grad) without arguments.  Returns (best shapes as a
    dict kernel -> (block, ctas_per_sm, chunk), report)."""
    ctx.tpc_profile_enable(True)
    best = {k: (0, 0, 0) for k in KERNELS}
    ctx.tpc_set_tuning(None)
    run()
    torch.cuda.synchronize()
    base = _stage_times(ctx, run, reps)
    report = {"default_stage_ms": base, "kernels": {}}
    for name in KERNELS:
        cand = candidates.get(name)
        if not cand:
            continue
        results = []
        for b in cand["block"]:
            for c in cand["ctas"]:
                for h in cand["chunk"]:
                    trial = dict(best)
                    trial[name] = (b, c, h)
                    ctx.tpc_set_tuning(to_struct(trial))
                    run()                                   # capture / warm
                    torch.cuda.synchronize()
                    st = ctx.tpc_sync_status()
                    if st != 0:
                        raise RuntimeError("device status %d while tuning %s" % (st, name))
                    t = _stage_times(ctx, run, reps)[name]
                    results.append((t, (b, c, h)))
        results.sort()
        default_t = base[name]
        t_best, shape = results[0]
        if t_best < default_t:
            best[name] = shape
        report["kernels"][name] = {"default_ms": default_t, "best_ms": min(t_best, default_t),
                                   "best": list(best[name]), "tried": len(results)}
        if log:
            log("tune %-10s default %.3f ms  best %.3f ms  %s" % (name, default_t, t_best, shape))
    ctx.tpc_set_tuning(to_struct(best))
    run()
    torch.cuda.synchronize()
    report["tuned_stage_ms"] = _stage_times(ctx, run, reps)
    ctx.tpc_profile_enable(False)
    return best, report
