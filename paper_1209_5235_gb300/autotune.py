"""Schedule and launch-shape autotuner of the transport.

Results never depend on the schedule (the persistent kernel or the staged
queues), the launch shape (block size, blocks per SM, the warp refill and
interaction thresholds, the voxel-walk budget per round, the period of
block-wide regrouping, the staged schedule's drain point) or the precision mode,
only speed does.  The tuner times trial launches of the caller's batch with CUDA
events: a few staged shapes, then the persistent kernel's parameters one at a
time from the defaults, keeping any value that is faster (coordinate descent),
within a time budget; a batch tuned on a proportional subset has its staged winner and that shape's
twin with the other relocation-kernel setting timed once more on the whole batch.  It only calls the
C ABI through the binding.
"""
from __future__ import annotations

import ctypes
import itertools
import time

from . import binding as b

SPACE = {
    "walk_budget": (1 << 16, 4, 8, 32),
    "regroup_period": (1, 2, 4),
    "block_size": (64, 96, 128),
    "blocks_per_sm": (0, 2, 3),
    "refill_min": (4, 8, 12, 16, 20, 24),
    "interact_min": (4, 8, 12, 16, 20, 24),
}
DEFAULT = {"block_size": 128, "blocks_per_sm": 0, "refill_min": 8, "interact_min": 8, "walk_budget": 16,
           "regroup_period": 0, "schedule": b.G4N_SCHEDULE_PERSISTENT, "pool_tracks": 0, "drain_tracks": 0,
           "staged_flags": 0}
# staged shapes tried: grids of one, two and four waves of the blocks that fit, with and without the separate
# relocation kernel; the drain at its default point, never, or early
STAGED = tuple({"drain_tracks": 0, "blocks_per_sm": bps, "staged_flags": fl}
               for fl in (0, b.G4N_STAGED_RELOCATION_KERNEL) for bps in (0, 8, 16)) + \
    ({"drain_tracks": -1, "blocks_per_sm": 0, "staged_flags": 0},
     {"drain_tracks": 1 << 20, "blocks_per_sm": 0, "staged_flags": 0})


def time_launch(ctx, items, seed, edep, cnt, mode, cfg, reps=2, stream=None):
    """Median device time (ms) of `reps` launches with launch shape `cfg`."""
    import torch
    st = stream or torch.cuda.current_stream()
    ts = []
    for r in range(reps):
        edep.zero_()
        cnt.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        b.g4n_transport_batch(ctx, items, seed + r, edep, cnt, n_batches=edep.shape[0], mode=mode, stream=st, **cfg)
        e1.record(st)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    b.g4n_sync(ctx, st)
    ts.sort()
    return ts[len(ts) // 2]


def subset_items(items, max_tracks):
    """The batch's items with their track counts scaled down to about `max_tracks` in total
    (every non-empty item keeps at least one track; ids and tally columns unchanged)."""
    total = sum(int(w.n_tracks) for w in items)
    if max_tracks <= 0 or total <= max_tracks:
        return items
    out = (b.g4n_work_item * len(items))()
    for k, w in enumerate(items):
        ctypes.pointer(out[k])[0] = w
        if w.n_tracks > 0:
            out[k].n_tracks = max(1, int(w.n_tracks) * max_tracks // total)
    return out


def autotune(ctx, items, stride, seed, modes=(b.G4N_MODE_FP64, b.G4N_MODE_FP32_RECHECK), n_batches=100, reps=2,
             budget_s=30.0, space=None, stream=None, max_tracks=2_000_000,
             schedules=(b.G4N_SCHEDULE_STAGED, b.G4N_SCHEDULE_PERSISTENT)):
    """Best (mode, schedule and launch shape) for the batch; returns dict(mode, cfg, ms, per_mode, trials).
    Batches of more than `max_tracks` tracks are tuned on a proportional subset (shorter
    trials, so that the budget covers the whole search)."""
    import torch
    space = space or SPACE
    full_items = items
    items = subset_items(items, max_tracks)
    edep = torch.zeros((n_batches, stride), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(b.G4N_N_COUNTERS, dtype=torch.int64, device="cuda")
    trials = []
    per_mode = {}
    for mode in modes:
        t_end = time.perf_counter() + budget_s / len(modes)   # each mode gets its share of the budget
        time_launch(ctx, items, seed, edep, cnt, mode, DEFAULT, reps=1, stream=stream)   # warm-up
        cfg, best = None, float("inf")
        if b.G4N_SCHEDULE_STAGED in schedules:
            for shape in STAGED:
                trial = dict(DEFAULT, schedule=b.G4N_SCHEDULE_STAGED, **shape)
                ms = time_launch(ctx, items, seed, edep, cnt, mode, trial, reps, stream)
                trials.append((mode, dict(trial), ms))
                if ms < best:
                    best, cfg = ms, trial
        if b.G4N_SCHEDULE_PERSISTENT not in schedules:
            per_mode[mode] = {"cfg": cfg, "ms": best}
            continue
        pcfg = dict(DEFAULT)
        pbest = time_launch(ctx, items, seed, edep, cnt, mode, pcfg, reps, stream)
        trials.append((mode, dict(pcfg), pbest))
        if pbest < best:
            best, cfg = pbest, pcfg
        for key in space:
            for val in space[key]:
                if val == pcfg[key] or time.perf_counter() > t_end:
                    continue
                trial = dict(pcfg, **{key: val})
                ms = time_launch(ctx, items, seed, edep, cnt, mode, trial, reps, stream)
                trials.append((mode, dict(trial), ms))
                if ms < pbest:
                    pbest, pcfg = ms, trial
                if ms < best:
                    best, cfg = ms, trial
        if items is not full_items and cfg["schedule"] == b.G4N_SCHEDULE_STAGED:
            # the staged kernels' balance shifts with the batch size: the winner and its relocation-kernel twin
            # are timed once more on the whole batch
            twin = dict(cfg, staged_flags=cfg["staged_flags"] ^ b.G4N_STAGED_RELOCATION_KERNEL)
            time_launch(ctx, full_items, seed, edep, cnt, mode, cfg, 1, stream)   # warm-up (the queues grow)
            full = {k: time_launch(ctx, full_items, seed, edep, cnt, mode, c, 1, stream)
                    for k, c in (("best", cfg), ("twin", twin))}
            trials.append((mode, dict(twin), full["twin"]))
            if full["twin"] < full["best"]:
                cfg = twin
            best = min(full.values()) * best / max(full["best"], 1e-9)   # keep the subset's scale for the ranking
        per_mode[mode] = {"cfg": cfg, "ms": best}
    mode = min(per_mode, key=lambda m: per_mode[m]["ms"])
    return {"mode": mode, "cfg": per_mode[mode]["cfg"], "ms": per_mode[mode]["ms"], "per_mode": per_mode,
            "trials": len(trials)}
