"""Autotuner for the coarse-peel schedule and the batch size.

The tip decomposition has knobs that change only how the work is laid out on
the GPU, never the tip numbers (every active vertex is still peeled with the
same supports, Sec. 3.1; any bounds give the same numbers, Th. 2):

- ``graph_rounds``: coarse rounds as one CUDA graph per range (device loop);
- ``warp_max_w`` / ``group_max_w``: wedge limits of the warp and 256-thread
  group classes of active vertices (the rest go to blocks);
- ``item_w``: wedges per block work item (splitting of heavy vertices);
- ``bucket_shift``: width 2^shift of the target-id buckets of block items;
- ``count_scratch``: scratch counters of the heavier counting starts
  (automatic, shared hashes first, dense shared label chunks);
- ``fd_cluster_min``: smallest fine-phase partition peeled by a
  thread-block cluster instead of one block (0 = the default 32768).

The tuner times candidate schedules on the caller's graph with CUDA events and
keeps the fastest, searching one knob at a time from the defaults (coordinate
descent: about a dozen runs instead of the full product).  ``tune_batch``
picks how many graphs go into one batched call.  Results can be cached in a
JSON file keyed by a signature of the graph (sizes and degree histogram).
"""
from __future__ import annotations

import json
import os
import time

DEFAULT = {"graph_rounds": False, "warp_max_w": 0, "group_max_w": 0, "item_w": 0, "bucket_shift": 0,
           "count_scratch": 0, "fd_cluster_min": 0}

# candidate values per knob (0 = the library's default)
SPACE = {
    "graph_rounds": [False, True],
    "warp_max_w": [0, 256, 128],
    "group_max_w": [0, 1024, 512],
    "item_w": [0, 8192, 131072],
    "bucket_shift": [0, 14, 16],
    "count_scratch": [0, 1, 2],
    "fd_cluster_min": [0, 8192, 0xFFFFFFFF],
}

WARP_MAX, GROUP_MAX = 512, 2048  # the library's limits (include/pbng.h)


def effective(cfg):
    """(warp limit, group limit) that the library will use for cfg."""
    wm = cfg.get("warp_max_w") or WARP_MAX
    gm = cfg.get("group_max_w") or GROUP_MAX
    return wm, gm


def valid(cfg):
    wm, gm = effective(cfg)
    iw = cfg.get("item_w") or 0
    sh = cfg.get("bucket_shift") or 0
    cs = cfg.get("count_scratch") or 0
    return (wm <= WARP_MAX and gm <= GROUP_MAX and wm <= gm and (iw == 0 or iw >= 4096) and (sh == 0 or 14 <= sh <= 30)
            and 0 <= cs <= 3)


def coordinate_search(measure, space=None, start=None, rounds=1):
    """Greedy coordinate descent over `space` from `start`.

    measure(cfg) -> seconds (smaller is better).  Returns (best cfg, its
    time, table of every (cfg, time) measured)."""
    space = SPACE if space is None else space
    best = dict(DEFAULT if start is None else start)
    best_t = measure(best)
    table = [(dict(best), best_t)]
    for _ in range(rounds):
        for k, vals in space.items():
            for v in vals:
                if best.get(k) == v:
                    continue
                c = dict(best)
                c[k] = v
                if not valid(c):
                    continue
                t = measure(c)
                table.append((dict(c), t))
                if t < best_t:
                    best, best_t = c, t
    return best, best_t, table


def split(cfg):
    """(keyword arguments of tip_decompose) for a schedule cfg."""
    sched = {k: int(cfg.get(k) or 0) for k in ("warp_max_w", "group_max_w", "item_w", "count_scratch", "fd_cluster_min")}
    return {"graph_rounds": bool(cfg.get("graph_rounds")), "bucket_shift": int(cfg.get("bucket_shift") or 0),
            "schedule": sched}


def signature(dg, side, P):
    """Sizes plus the log2 degree histogram of the U side (computed on the device)."""
    import torch
    off = dg.u_off.to(torch.int64)
    du = (off[1:] - off[:-1]).clamp(min=1)
    h = torch.bincount(torch.log2(du.double()).floor().to(torch.int64), minlength=32)[:32].tolist()
    return f"{dg.nu}x{dg.nv}x{dg.m}:{side}:{P}:" + ",".join(str(int(x)) for x in h)


def _time(fn, reps):
    import torch
    best = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1000.0)
    return best


def tune_tip(dg, side="U", P=150, reps=2, space=None, cache=None, rounds=1):
    """Fastest schedule for tip_decompose(dg, side, P); (cfg, seconds, table).

    cache: optional JSON path; a stored result for the same signature is
    returned without measuring."""
    from . import tip_decompose
    key = signature(dg, side, P)
    if cache and os.path.exists(cache):
        with open(cache) as f:
            stored = json.load(f)
        if key in stored:
            r = stored[key]
            return r["cfg"], r["seconds"], []
    tip_decompose(dg, side, P=P)  # warm the library's pool

    def measure(cfg):
        kw = split(cfg)
        return _time(lambda: tip_decompose(dg, side, P=P, **kw), reps)

    best, t, table = coordinate_search(measure, space, rounds=rounds)
    if cache:
        stored = {}
        if os.path.exists(cache):
            with open(cache) as f:
                stored = json.load(f)
        stored[key] = {"cfg": best, "seconds": t, "when": time.time()}
        with open(cache, "w") as f:
            json.dump(stored, f, indent=1)
    return best, t, table


def tune_batch_schedule(dgs, side="U", P=150, sample=512, reps=1, space=None):
    """Schedule for batched calls, timed on the first `sample` graphs."""
    from . import tip_decompose_batch
    part = dgs[:sample]
    tip_decompose_batch(part, side, P=P)

    def measure(cfg):
        kw = split(cfg)
        return _time(lambda: tip_decompose_batch(part, side, P=P, **kw), reps)

    return coordinate_search(measure, space)


def tune_batch(dgs, side="U", P=150, sizes=(256, 1024, 4096), reps=1, cfg=None):
    """Graphs per batched call with the best throughput; (size, table)."""
    from . import tip_decompose_batch
    kw = split(cfg or DEFAULT)
    table = []
    for s in sizes:
        s = max(1, min(s, len(dgs)))

        def run():
            for i in range(0, len(dgs), s):
                tip_decompose_batch(dgs[i:i + s], side, P=P, **kw)

        run()
        table.append((s, _time(run, reps)))
    best = min(table, key=lambda r: r[1])[0]
    return best, table
