"""Autotuner: picks kernel variants and launch shapes by measurement.

The paper names "an automatic scheduler for hardware-specific optimal
performance" as future work (Sec. VI). Here the library exposes its choices as
explicit variant codes (rnea_batch: per-thread serial recursion in joint frames
with one of four backward-state modes -- stored, stateless, cos/sin only, or
stored for the first K links -- and a block size; the same in common-normal
frames with the constants as a kernel parameter and K stored links, or with
the state of the first links in tensor memory; or the lane-parallel scan with L
lanes; fleet_batch: persistent CTA shape or one launch per group), and this
module times the candidates on the caller's own data with CUDA events, keeps
the fastest, and caches the answer in a JSON file keyed by GPU name, SM count
and the workload's shape (RDYN_TUNE_CACHE, default ~/.cache/rdyn/tune.json).
It only times library calls; it computes nothing itself.
"""
from __future__ import annotations

import json
import os
import threading

from . import binding as b

_lock = threading.Lock()


def cache_path():
    return os.environ.get("RDYN_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "rdyn", "tune.json"))


def _load_cache():
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(key, value):
    with _lock:
        c = _load_cache()
        c[key] = value
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(c, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _gpu_key(torch, dev):
    p = torch.cuda.get_device_properties(dev)
    return f"{p.name}|{p.multi_processor_count}"


def _time(torch, fn, reps=5):
    """Median of `reps` timings (ms) of fn() after one warm-up, CUDA events on the
    current stream."""
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    return ts[len(ts) // 2]


def rnea_candidates(n, B, dtype):
    c = [b.RD_VARIANT_AUTO]
    for block in (32, 64, 128):
        for mode in (b.RD_VARIANT_SERIAL, b.RD_VARIANT_SERIAL_RECOMPUTE,
                     b.RD_VARIANT_SERIAL_RECOMPUTE_CS):
            c.append(mode | b.RD_TUNE_BLOCK(block))
    for block in (32, 64):  # state for the first K links only
        for K in (4, 8, 12, 16, 24):
            if K < n:
                c.append(b.RD_VARIANT_SERIAL_HYBRID | b.RD_TUNE_STORED_LINKS(K) |
                         b.RD_TUNE_BLOCK(block))
    # common-normal frames: full state for the first K links (0 = library default)
    for block in (32, 64):
        c.append(b.RD_VARIANT_SERIAL_DH_RECOMPUTE | b.RD_TUNE_BLOCK(block))
        for K in (0, 8, 12, 16, 20, 24, 32):
            if K <= n:
                c.append(b.RD_VARIANT_SERIAL_DH | b.RD_TUNE_STORED_LINKS(K) |
                         b.RD_TUNE_BLOCK(block))
    if n <= 32 and n % 4 == 0 and str(dtype) in ("torch.float32", "float32", "None"):
        for K in (0, 16, 20, 24):  # state of the first links in tensor memory
            if K <= n:
                c.append(b.RD_VARIANT_SERIAL_DH_TMEM | b.RD_TUNE_STORED_LINKS(K))
    for lanes in (2, 4, 8, 16, 32):
        if n <= 8 * lanes:
            c.append(b.RD_VARIANT_SCAN(lanes))
    return c


def tune_rnea(model, q, qd, qdd, out=None, reps=5, use_cache=True):
    """Fastest rnea_batch variant for this (model length, batch, dtype); returns
    (variant, {variant: ms})."""
    import torch

    key = f"rnea|{_gpu_key(torch, q.device)}|n={model.n}|B={q.shape[0]}|{q.dtype}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit is not None:
            return int(hit["variant"]), hit.get("times", {})
    out = out if out is not None else torch.empty_like(q)
    times = {}
    for v in rnea_candidates(model.n, q.shape[0], q.dtype):
        try:
            times[v] = _time(torch, lambda: b.rnea(model, q, qd, qdd, out=out, variant=v), reps)
        except b.RdError:
            continue
    best = min(times, key=times.get)
    _store(key, {"variant": best, "times": {str(k): t for k, t in times.items()}})
    return best, times


def fleet_candidates():
    """(schedule, tune) pairs: one launch per group; the persistent kernel at
    several block shapes with one thread per request; and the persistent kernel
    with two or three warps per 32 forward-dynamics requests for the groups whose
    chains reach a threshold (the warps per request of each n-range)."""
    c = [(b.RD_SCHED_PER_GROUP, 0)]
    for lt in (5, 6, 7, 8):
        for per_sm in (1, 2, 4, 8):
            if (1 << lt) * per_sm <= 1024:
                c.append((b.RD_SCHED_PERSISTENT, b.RD_FLEET_TUNE(lt, per_sm)))
    for min_links in (6, 33, 65):
        for lt in (6, 7, 8):
            for per_sm in (1, 2, 4):
                if (1 << lt) * per_sm <= 1024:
                    c.append((b.RD_SCHED_PERSISTENT,
                              b.RD_FLEET_TUNE(lt, per_sm) | b.RD_FLEET_TWO_WARPS(min_links)))
    for min_links in (33, 65):
        for lt in (6, 7):
            for per_sm in (1, 2, 4):
                c.append((b.RD_SCHED_PERSISTENT,
                          b.RD_FLEET_TUNE(lt, per_sm) | b.RD_FLEET_THREE_WARPS(min_links)))
    return c


def tune_fleet(plan, q, qd, in2, out=None, reps=3, use_cache=True, flags=0):
    """Fastest (schedule, tune word) for this plan's request mix, every candidate
    run with ``flags`` (e.g. RD_FLEET_FP64_UPDATE) OR-ed into its schedule;
    returns ((schedule, tune), {(schedule, tune): ms}) without the flags."""
    import zlib

    import numpy as np
    import torch

    hist = np.bincount(plan.lengths * 2 + plan.kinds, minlength=2 * 130)
    sig = (f"R={plan.R}|J={plan.total_joints}|h={zlib.crc32(hist.tobytes()):08x}|{plan.dtype}"
           f"|f={int(flags):x}")
    key = f"fleet|{_gpu_key(torch, q.device)}|{sig}"
    if use_cache:
        hit = _load_cache().get(key)
        if hit is not None:
            return (int(hit["schedule"]), int(hit["tune"])), {}
    out = out if out is not None else torch.empty_like(q)
    times = {}
    for sched, tune in fleet_candidates():
        times[(sched, tune)] = _time(
            torch, lambda: b.fleet_batch(plan, q, qd, in2, out=out, schedule=sched | flags,
                                         tune=tune), reps)
    best = min(times, key=times.get)
    _store(key, {"schedule": best[0], "tune": best[1],
                 "times": {f"{k[0]}:{k[1]}": t for k, t in times.items()}})
    return best, times
