"""Launch-shape autotuner.

Every option it touches chooses among kernels that compute identical values
(the per-sample arithmetic, including the lane grouping of the network, is
fixed per width), so tuning changes speed only.  It times each candidate on
the caller's own workload with CUDA events on the launching stream and
applies the fastest:

* plan steps: the collision-kernel variant (block-balanced, warp items,
  point-sliced items with 2 or 4 warps) for a given (width, N, T, M);
* batches: the number of warps sharing one 8-sample collision item (the
  obstacle-point slice each warp checks) and the warps per trajectory block
  (samples per block).

Results are cached per workload key in memory and, when `path` is given, in
a JSON file.
"""
import json
import os

import numpy as np
import torch

from . import npp

PLAN_VARIANTS = (0, 1, 2, 3, 4)
# (collision check, point slices, trajectory warps): check 1 = per-step bins
# (slices unused), 0 = brute force over cell-sorted point tiles
BATCH_CANDIDATES = tuple([(1, 4, w) for w in (4, 8)] + [(0, s, w) for s in (2, 4, 8) for w in (4, 8)])

_cache = {}


def _load(path):
    if path and os.path.exists(path):
        try:
            _cache.update(json.load(open(path)))
        except (OSError, ValueError):
            pass


def _store(path):
    if path:
        tmp = path + ".tmp"
        json.dump(_cache, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, path)


def plan_key(width, N, T, M):
    """Bucket: width, N and M rounded to powers of two, T to multiples of 10."""
    b = lambda x: int(2 ** round(np.log2(max(1, x))))
    return "plan:w%d:N%d:T%d:M%d" % (width, b(N), 10 * max(1, round(T / 10)), b(M))


def tune_plan_step(planner, state, goal, obs, N, T, seed, reps=3, path=None):
    """Pick the collision variant for this workload; returns (variant, ms per
    variant).  `planner` is an npp.Planner; obs a CUDA tensor [M, 4]."""
    _load(path)
    M = 0 if obs is None else obs.shape[0]
    key = plan_key(planner.cfg.width, N, T, M)
    if key in _cache:
        v = int(_cache[key]["variant"])
        npp.npp_set_option(planner.h, "collide_variant", v)
        return v, _cache[key]["ms"]
    npp.npp_set_timing(planner.h, True)
    times = {}
    for v in PLAN_VARIANTS:
        npp.npp_set_option(planner.h, "collide_variant", v)
        ts = []
        for r in range(reps + 1):
            planner.plan(state, goal, obs, N, T, seed, r)
            ts.append(npp.npp_last_timing(planner.h)["collide"])
        times[v] = float(np.median(ts[1:]))
    best = min(times, key=times.get)
    npp.npp_set_option(planner.h, "collide_variant", best)
    _cache[key] = {"variant": best, "ms": {str(k): v for k, v in times.items()}}
    _store(path)
    return best, _cache[key]["ms"]


def _set_batch(batch, cand):
    c, s, w = cand
    npp.npp_batch_set_option(batch, "collide", c)
    npp.npp_batch_set_option(batch, "slices", s)
    npp.npp_batch_set_option(batch, "traj_warps", w)


def tune_batch(batch, obs, out, key, reps=2, path=None, stream=None):
    """Pick (collision check, slices, traj_warps) for a batch; returns the
    choice and ms per candidate.  `key` names the batch layout for the
    cache."""
    _load(path)
    k = "batch:" + key
    if k in _cache and len(_cache[k]["best"]) == 3:
        best = tuple(_cache[k]["best"])
        _set_batch(batch, best)
        return best, _cache[k]["ms"]
    stream = stream or torch.cuda.current_stream()
    times = {}
    for cand in BATCH_CANDIDATES:
        _set_batch(batch, cand)
        ts = []
        for r in range(reps + 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            npp.npp_plan_batch(batch, obs, out, stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        times[cand] = float(np.median(ts[1:]))
    best = min(times, key=times.get)
    _set_batch(batch, best)
    _cache[k] = {"best": list(best), "ms": {"%d,%d,%d" % c: t for c, t in times.items()}}
    _store(path)
    return best, _cache[k]["ms"]
