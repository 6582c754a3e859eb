#!/usr/bin/env python
"""Benchmark of the GB300 two-phase tip decomposition.

One step = plain GPU two-phase tip decomposition (PBNG, Sec. 3.1-3.2) of BOTH
vertex sides of the Chung-Lu power-law bipartite graph |U|=1M, |V|=200k,
m=20M, degree exponents 2.1 (U) and 2.5 (V), degree cap 50k, P=150, with
the graph resident in HBM.  Metric: wedges traversed per second (the
paper's work unit, Tab. 4) over the whole job; ms_per_step is the
decomposition time of both sides.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pbng|reference]

N > 1 (one process per GPU under torch.distributed.run): every rank
decomposes its own replica of the graph; there is no data-path collective.
--impl reference times the CPU oracle (sequential bottom-up peeling,
Alg. 2) on a bounded sample of the same workload (the same sample whatever
--steps is).

At N = 1 the line also carries the batched/learned comparison of the
metric, each measured with CUDA events in this process:
  batched: 4,096 independent graphs (batch workload) in one batched call
           vs the same graphs decomposed one call at a time;
  learned: tip decomposition of the 5M x 1M, 60M-edge Chung-Lu graph with
           the learned bound proposer vs the plain range estimator;
  wing:    wing decomposition of the planted 500k x 100k graph (P = 100).
Their inputs are generated by a process pool started before the first GPU
call, while the main workload is timed.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "chunglu_1m_200k_20m"
WORKLOAD_DESC = ("plain GPU two-phase tip decomposition of both sides, Chung-Lu |U|=1M |V|=200k m=20M, "
                 "exponents 2.1/2.5, degree cap 50k, P=150")
# CPU-baseline sample: the same Chung-Lu recipe at 1/20 scale
SAMPLE = dict(kind="chung_lu", nu=50000, nv=10000, m=1000000, gu=2.1, gv=2.5, dmax=5000, seed=22)
SAMPLE_DESC = "oracle BUP tip decomposition of both sides of the same Chung-Lu recipe at 1/20 scale (|U|=50k |V|=10k m=1M)"
# the oracle's complete tip peeling of both sides of the full graph, measured once on the
# build host when the expected results were written (tests/golden/*.json, cpu_seconds)
GOLDEN_SIDES = ("tip_chunglu_1m_200k_20m_U", "tip_chunglu_1m_200k_20m_V")
BATCH_N, BATCH_SEED0 = 4096, 1000
LEARNED_WORKLOAD, LEARNED_P = "chunglu_5m_1m_60m", 200
WING_WORKLOAD, WING_P = "chunglu_500k_100k_5m_planted", 100


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources each kernel group is compiled from
GROUP_SOURCES = {"peel": ("tip.cu", "wedge.cuh", "fdwin.cuh", "internal.cuh"),
                 "fd": ("tip.cu", "wedge.cuh", "fdwin.cuh", "internal.cuh"),
                 "count": ("count.cu", "wedge.cuh", "internal.cuh")}


def kernel_sources_sha(group):
    """Hash of the sources of one kernel group (a stored traffic figure is
    used only while they are unchanged)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2110_12511_gb300", "csrc")
    for n in GROUP_SOURCES[group]:
        h.update(open(os.path.join(d, n), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(group):
    """DRAM bytes per launch of a kernel group from the committed ncu summary,
    or None when the kernel sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    sha = kernel_sources_sha(group)
    for line in open(p):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == WORKLOAD and f[1] == group and f[2] == sha:
            return float(f[3])
    return None


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.lines = []

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.p = None
        return self

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """Largest value of a host float over all ranks (all_reduce MAX); x when ws == 1."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ws, seconds_max):
    """Units all ranks processed (each rank the same replica workload) per second of the slowest."""
    return ws * units_per_rank / seconds_max


def tip_wedges(st):
    return st["wedges_count"] + st["wedges_cd"] + st["wedges_fd"]


def oracle_sample(spec, sides=("U", "V")):
    """Time the oracle on a sample; returns (wedges, seconds).  The wedges are
    the ones the oracle's own loops visit, counted exactly: its 2-hop count
    visits sum_y d_y^2 wedges (y on the other side) and its peel visits every
    wedge of each peeled vertex once more, so 2 sum_y d_y^2 per side."""
    import bigraph_gen as gen
    import oracle
    g = gen.make(dict(spec))
    du = np.diff(g.u_off).astype(np.float64)
    dv = np.bincount(g.u_adj, minlength=g.nv).astype(np.float64)
    t0 = time.perf_counter()
    for s in sides:
        oracle.tip(g, s)
    dt = time.perf_counter() - t0
    w = 0.0
    for s in sides:
        w += 2.0 * float((dv ** 2).sum() if s == "U" else (du ** 2).sum())
    return w, dt


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    spec, desc = SAMPLE, SAMPLE_DESC
    for _ in range(args.warmup):
        oracle_sample(spec)
    tw, tt = 0.0, 0.0
    for _ in range(args.steps):
        w, dt = oracle_sample(spec)
        tw += w
        tt += dt
    v = tw / tt
    line = {"metric": "tip decomposition wedges/s (both sides)", "value": v, "unit": "wedges/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD_DESC, "sample": desc},
            "cpu_baseline": {"value": v, "unit": "wedges/s", "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "wedges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed(fn, dev, flush):
    """Device time of fn() in ms with the L2 flushed first."""
    import torch
    flush.zero_()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1), out


def run_extra(args):
    """Measurements of the other workloads (not the default bench line)."""
    import torch
    import bigraph_gen as gen
    import paper_2110_12511_gb300 as pbng
    from paper_2110_12511_gb300 import build as pbuild
    pbuild.build()
    pbng.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    res = {"workload": args.workload}
    if args.workload == "wing_chunglu_500k_100k_5m_planted":
        t0 = time.time()
        g = gen.make("chunglu_500k_100k_5m_planted")
        res["gen_s"] = time.time() - t0
        dg = pbng.to_device(g, dev)
        P = 100
        for _ in range(args.warmup):
            pbng.wing_decompose(dg, P=P)
        ms, st = [], None
        for _ in range(args.steps):
            t, (_, st) = timed(lambda: pbng.wing_decompose(dg, P=P, with_stats=True), dev, flush)
            ms.append(t)
        res.update({"m": g.m, "P": P, "ms": statistics.median(ms), "ms_all": ms,
                    "updates_per_s": st["updates"] / (statistics.median(ms) / 1e3),
                    "links_traversed_per_s": (st["wedges_cd"] + st["wedges_fd"]) / (statistics.median(ms) / 1e3),
                    "stats": st})
    elif args.workload == "tip_batch_4096":
        t0 = time.time()
        n = args.batch
        gs = [gen.batch_graph(1000 + i) for i in range(n)]
        res["gen_s"] = time.time() - t0
        dgs = [pbng.to_device(g, dev) for g in gs]
        res.update({"graphs": n, "edges": int(sum(g.m for g in gs))})
        P = 150
        bkw, size = {}, n
        if args.autotune:  # schedule on a sample, then the batch size (not timed)
            from paper_2110_12511_gb300 import autotune
            cfg, _, _ = autotune.tune_batch_schedule(dgs, "U", P=P)
            size, _ = autotune.tune_batch(dgs, "U", P=P, sizes=(1024, 2048, n), cfg=cfg)
            bkw = autotune.split(cfg)
            res.update({"schedule": cfg, "batch_size": size})
        elif args.graph_rounds:
            bkw = {"graph_rounds": True}
            res["schedule"] = bkw

        def batched():
            stats = None
            for i in range(0, n, size):
                _, s1 = pbng.tip_decompose_batch(dgs[i:i + size], "U", P=P, with_stats=True, **bkw)
                stats = s1 if stats is None else {k: stats[k] + s1[k] for k in ("wedges_count", "wedges_cd", "wedges_fd")}
            return None, stats

        batched()
        tb, (_, stb) = timed(batched, dev, flush)
        def one_by_one():
            w = 0
            for d in dgs:
                _, s1 = pbng.tip_decompose(d, "U", P=P, with_stats=True)
                w += s1["wedges_count"] + s1["wedges_cd"] + s1["wedges_fd"]
            return w
        one_by_one_w = one_by_one() if n <= 64 else None
        tp, wp = timed(one_by_one, dev, flush)
        res.update({"P": P, "batched_ms": tb, "plain_one_by_one_ms": tp, "speedup": tp / tb,
                    "batched_wedges_per_s": (stb["wedges_count"] + stb["wedges_cd"] + stb["wedges_fd"]) / (tb / 1e3),
                    "batched_stats": stb, "plain_wedges": wp})
    elif args.workload == "tip_chunglu_5m_1m_60m":
        t0 = time.time()
        g = gen.make("chunglu_5m_1m_60m")
        res["gen_s"] = time.time() - t0
        dg = pbng.to_device(g, dev)
        P = 200
        pbng.tip_decompose(dg, "U", P=P, graph_rounds=args.graph_rounds)
        t, (_, st) = timed(lambda: pbng.tip_decompose(dg, "U", P=P, with_stats=True, graph_rounds=args.graph_rounds),
                           dev, flush)
        res.update({"m": g.m, "P": P, "ms": t, "graph_rounds": args.graph_rounds, "wedges_per_s": (st["wedges_count"] + st["wedges_cd"] + st["wedges_fd"]) / (t / 1e3),
                    "stats": st})
    elif args.workload == "tip_uniform_2k_1k_20k":
        g = gen.make("uniform_2k_1k_20k")
        dg = pbng.to_device(g, dev)
        P = 8
        kw = {"graph_rounds": args.graph_rounds}
        for _ in range(max(args.warmup, 3)):
            pbng.tip_decompose(dg, "U", P=P, **kw)
        ms = []
        for _ in range(max(args.steps, 20)):
            t, (_, st) = timed(lambda: pbng.tip_decompose(dg, "U", P=P, with_stats=True, **kw), dev, flush)
            ms.append(t)
        h = gen.make("uniform_2k_1k_20k")
        e2e = []
        for _ in range(max(args.steps, 20)):
            t0 = time.perf_counter()
            pbng.tip_decompose_host(h, "U", P=P, **kw)
            e2e.append((time.perf_counter() - t0) * 1e3)
        res.update({"m": g.m, "P": P, "ms_median": statistics.median(ms), "e2e_host_buffers_ms_median": statistics.median(e2e),
                    "graph_rounds": args.graph_rounds, "stats": st})
    elif args.workload == "tip_chunglu_5m_1m_60m_learned":
        from paper_2110_12511_gb300 import learned
        g = gen.make("chunglu_5m_1m_60m")
        dg = pbng.to_device(g, dev)
        P = 200
        mlp = learned.load()
        out = {}
        ref = None
        for mode in ("estimator", "learned", "estimator", "learned"):
            kw = {"mlp": mlp} if mode == "learned" else {}
            t, (th, st) = timed(lambda: pbng.tip_decompose(dg, "U", P=P, with_stats=True, **kw), dev, flush)
            th = pbng.as_u64(th)
            if ref is None:
                ref = th
            assert (th == ref).all(), "learned bounds changed the tip numbers"
            r = out.setdefault(mode, {"ms": []})
            r["ms"].append(t)
            r.update({k: st[k] for k in ("rounds", "parts_used", "launches", "fd_work_max", "fd_work_sum", "wedges_cd")})
        for r in out.values():
            r["best_ms"] = min(r["ms"])
            r["fd_imbalance"] = r["fd_work_max"] / max(1.0, r["fd_work_sum"] / max(1, r["parts_used"]))
        res.update({"P": P, "identical_theta": True, **out,
                    "learned_speedup": out["estimator"]["best_ms"] / out["learned"]["best_ms"]})
    elif args.workload == "tip_components":
        # k-tips of both sides of the 1M x 200k graph at the median and the 99th
        # percentile tip number (tip numbers from the decomposition, not timed)
        g = gen.make(WORKLOAD)
        dg = pbng.to_device(g, dev)
        for side in ("U", "V"):
            th = pbng.tip_decompose(dg, side, P=args.P)
            thn = pbng.as_u64(th)
            out = {}
            for q in (50, 99):
                k = int(np.percentile(thn, q))
                pbng.tip_components(dg, side, th, k)
                t, (comp, st) = timed(lambda: pbng.tip_components(dg, side, th, k, with_stats=True), dev, flush)
                c = comp.cpu().numpy().view(np.uint32)
                mem = c != 0xFFFFFFFF
                out[f"p{q}"] = {"k": k, "ms": t, "members": int(mem.sum()), "tips": int(len(np.unique(c[mem]))),
                                "wedges": st["wedges_fd"], "pairs": st["updates"]}
            res[side] = out
    elif args.workload in ("tip_ablation", "tip_p_sweep"):
        g = gen.make(WORKLOAD)
        dg = pbng.to_device(g, dev)

        def run(side, P, **kw):
            pbng.tip_decompose(dg, side, P=P, **kw)  # warm
            t, (_, st) = timed(lambda: pbng.tip_decompose(dg, side, P=P, with_stats=True, **kw), dev, flush)
            return {"ms": t, "wedges_cd": st["wedges_cd"], "wedges_fd": st["wedges_fd"], "updates": st["updates"],
                    "rounds": st["rounds"], "recounts": st["recounts"], "parts_used": st["parts_used"],
                    "phase_ms": {k: st["ns_" + k] / 1e6 for k in ("count", "cd", "part", "fd")},
                    "fd_work_max": st["fd_work_max"], "fd_work_sum": st["fd_work_sum"]}

        if args.workload == "tip_ablation":
            # Sec. 6 ablations: PBNG, PBNG- (no dynamic graph updates), PBNG-- (neither dynamic
            # updates nor batched re-counting); host-driven rounds (the re-count branch)
            variants = {"PBNG": {}, "PBNG-": {"compact": False}, "PBNG--": {"compact": False, "recount": False}}
            for side in ("U", "V"):
                res[side] = {name: run(side, args.P, **kw) for name, kw in variants.items()}
        else:  # partition count sweep, both sides, default configuration
            for side in ("U", "V"):
                res[side] = {str(P): run(side, P) for P in (10, 50, 150, 400, 1000)}
    elif args.workload in ("wing_ablation", "wing_p_sweep", "wing_learned"):
        g = gen.make(WING_WORKLOAD)
        dg = pbng.to_device(g, dev)

        def run_w(P, **kw):
            pbng.wing_decompose(dg, P=P, **kw)  # warm
            t, (th, st) = timed(lambda: pbng.wing_decompose(dg, P=P, with_stats=True, **kw), dev, flush)
            return th, {"ms": t, "links": st["links"], "updates": st["updates"], "rounds": st["rounds"],
                        "parts_used": st["parts_used"], "fd_steps_max": st["fd_part_steps_max"],
                        "phase_ms": {k: st["ns_" + k] / 1e6 for k in ("count", "cd", "part", "fd")},
                        "fd_work_max": st["fd_work_max"], "fd_work_sum": st["fd_work_sum"]}

        res["m"] = g.m
        if args.workload == "wing_ablation":
            # Sec. 6 ablations for wing: PBNG, PBNG- (no dynamic BE-Index updates:
            # pair lists are never compacted)
            ref = None
            for name, kw in {"PBNG": {}, "PBNG-": {"compact": False}}.items():
                th, res[name] = run_w(WING_P, **kw)
                th = pbng.as_u64(th)
                ref = th if ref is None else ref
                assert (th == ref).all(), "ablation changed the wing numbers"
        elif args.workload == "wing_p_sweep":
            for P in (25, 50, 100, 200, 400, 1000):
                res[str(P)] = run_w(P)[1]
        else:  # learned wing bounds against the estimator (judged by default, and unjudged)
            from paper_2110_12511_gb300 import learned
            mlp = learned.load(learned.WING_WEIGHTS, device=dev)
            ref = None
            for name, kw in {"estimator": {}, "learned": {"mlp": mlp}, "learned_unjudged":
                             {"mlp": mlp, "learned_vet": -1.0}}.items():
                best = None
                for _ in range(2):
                    th, r = run_w(WING_P, **kw)
                    best = r if best is None or r["ms"] < best["ms"] else best
                th = pbng.as_u64(th)
                ref = th if ref is None else ref
                assert (th == ref).all(), "learned bounds changed the wing numbers"
                res[name] = best
            res["ratio"] = res["estimator"]["ms"] / res["learned"]["ms"]
            res["ratio_unjudged"] = res["estimator"]["ms"] / res["learned_unjudged"]["ms"]
    else:
        raise SystemExit(f"unknown workload {args.workload}")
    print(json.dumps(res), flush=True)
    return 0


def _gen_worker(job):
    """One input of the bench, generated in a spawned worker process (no GPU)."""
    import bigraph_gen as gen
    kind, a, b = job
    if kind == "batch":
        return [gen.batch_graph(s) for s in range(a, b)]
    return gen.make(a)


def start_inputs(extras):
    """Spawned pool generating the main workload and, with extras, the inputs
    of the batched / learned / wing records (started before any GPU call)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(min(12, max(2, (os.cpu_count() or 2) - 1)))
    jobs = {"main": pool.apply_async(_gen_worker, (("make", WORKLOAD, 0),))}
    if extras:
        jobs["learned"] = pool.apply_async(_gen_worker, (("make", LEARNED_WORKLOAD, 0),))
        chunk = BATCH_N // 8
        jobs["batch"] = [pool.apply_async(_gen_worker, (("batch", BATCH_SEED0 + i, BATCH_SEED0 + i + chunk),))
                         for i in range(0, BATCH_N, chunk)]
        jobs["wing"] = pool.apply_async(_gen_worker, (("make", WING_WORKLOAD, 0),))
    return pool, jobs


def record_batched(pbng, graphs, dev, flush, P=150):
    """The batch workload in one batched call vs one call per graph, both with
    graph-captured coarse rounds, CUDA events on the library's stream."""
    import torch
    dgs = [pbng.to_device(g, dev) for g in graphs]
    kw = {"graph_rounds": True}
    pbng.tip_decompose_batch(dgs, "U", P=P, **kw)
    tb, (res, stb) = timed(lambda: pbng.tip_decompose_batch(dgs, "U", P=P, with_stats=True, **kw), dev, flush)
    for d in dgs[:16]:
        pbng.tip_decompose(d, "U", P=P, **kw)
    to, outs = timed(lambda: [pbng.tip_decompose(d, "U", P=P, **kw) for d in dgs], dev, flush)
    same = all(torch.equal(a, b) for a, b in zip(res, outs))
    assert same, "batched and one-at-a-time tip numbers differ"
    w = tip_wedges(stb)
    return {"workload": f"tip decomposition (U, P={P}) of {len(graphs)} Chung-Lu graphs with planted bicliques, "
                        "m log-uniform in 1k-200k", "graphs": len(graphs), "edges": int(sum(g.m for g in graphs)),
            "batched_ms": tb, "one_at_a_time_ms": to, "ratio": to / tb, "identical_theta": same,
            "batched_wedges_per_s": w / (tb / 1e3), "rounds": stb["rounds"], "parts_used": stb["parts_used"],
            "mode": "graph-captured coarse rounds in both arms"}


def record_learned(pbng, g, dev, flush, P=LEARNED_P):
    """Learned bound proposer vs the plain range estimator on the 60M-edge graph."""
    from paper_2110_12511_gb300 import learned
    dg = pbng.to_device(g, dev)
    mlp = learned.load(device=dev)
    out, ref = {}, None
    for mode in ("estimator", "learned", "estimator", "learned"):
        kw = {"mlp": mlp} if mode == "learned" else {}
        t, (th, st) = timed(lambda: pbng.tip_decompose(dg, "U", P=P, with_stats=True, graph_rounds=True, **kw),
                            dev, flush)
        th = pbng.as_u64(th)
        if ref is None:
            ref = th
        assert (th == ref).all(), "learned bounds changed the tip numbers"
        r = out.setdefault(mode, {"ms": []})
        r["ms"].append(t)
        r.update({k: st[k] for k in ("rounds", "parts_used", "fd_work_max", "fd_work_sum", "wedges_cd", "wedges_fd")})
        r["phase_ms"] = {k: st["ns_" + k] / 1e6 for k in ("count", "cd", "part", "fd")}
    for r in out.values():
        r["best_ms"] = min(r["ms"])
        r["fd_imbalance"] = r["fd_work_max"] / max(1.0, r["fd_work_sum"] / max(1, r["parts_used"]))
    return {"workload": f"tip decomposition (U, P={P}) of Chung-Lu |U|=5M |V|=1M m=60M, exponents 2.1/2.3",
            "identical_theta": True, **out, "ratio": out["estimator"]["best_ms"] / out["learned"]["best_ms"]}


def record_wing(pbng, g, dev, flush, P=WING_P):
    """Wing decomposition of the planted 500k x 100k graph."""
    dg = pbng.to_device(g, dev)
    pbng.wing_decompose(dg, P=P)
    t, (_, st) = timed(lambda: pbng.wing_decompose(dg, P=P, with_stats=True), dev, flush)
    return {"workload": f"wing decomposition (P={P}) of Chung-Lu |U|=500k |V|=100k m=5M, exponents 2.2/2.4, "
                        "200 planted bicliques 20-200 x 20-200", "m": g.m, "ms": t,
            "updates_per_s": st["updates"] / (t / 1e3), "links": st["links"], "rounds": st["rounds"],
            "parts_used": st["parts_used"], "fd_steps_max": st["fd_part_steps_max"],
            "phase_ms": {k: st["ns_" + k] / 1e6 for k in ("count", "cd", "part", "fd")}}


def full_graph_oracle_seconds():
    """The oracle's measured time for the complete tip peeling of both sides of
    the full workload (written with the stored expected results), or None."""
    tot, hosts = 0.0, set()
    for name in GOLDEN_SIDES:
        p = os.path.join(ROOT, "tests", "golden", name + ".json")
        if not os.path.exists(p):
            return None
        with open(p) as f:
            d = json.load(f)
        tot += float(d["cpu_seconds"])
        hosts.add(d.get("host", "x86_64"))
    return {"seconds": tot, "host": ",".join(sorted(hosts)), "cores": 1}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pbng", choices=["pbng", "reference"])
    ap.add_argument("--P", type=int, default=150)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer run (profiling)")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="default: the bench line; others: tip_uniform_2k_1k_20k, wing_chunglu_500k_100k_5m_planted, "
                         "tip_batch_4096, tip_chunglu_5m_1m_60m, tip_chunglu_5m_1m_60m_learned, tip_ablation, "
                         "tip_p_sweep, tip_components, wing_ablation, wing_p_sweep, wing_learned")
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--host-rounds", dest="graph_rounds", action="store_false",
                    help="drive the coarse rounds from the host (default: one CUDA graph per range, device loop)")
    ap.add_argument("--no-recount", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the coarse-peel schedule per side with the autotuner before timing (not timed)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched / learned / wing records of the line")
    args = ap.parse_args()
    ws, rank, local = dist_info()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload != WORKLOAD:
        return run_extra(args)

    extras = ws == 1 and not args.no_extras
    pool, jobs = start_inputs(extras)  # before the first GPU call

    import torch
    import torch.distributed as dist
    import paper_2110_12511_gb300 as pbng
    from paper_2110_12511_gb300 import build as pbuild

    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or ws == 1:
        pbuild.build()
    if ws > 1:
        dist.barrier()
    pbng.lib()

    g = jobs["main"].get()
    dg = pbng.to_device(g, dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    kw = {"graph_rounds": args.graph_rounds, "recount": not args.no_recount}
    kws = {"U": dict(kw), "V": dict(kw)}
    tuned = None
    if args.autotune:
        from paper_2110_12511_gb300 import autotune
        tuned = {}
        for side in ("U", "V"):
            cfg, _, _ = autotune.tune_tip(dg, side, P=args.P, reps=1)
            tuned[side] = cfg
            kws[side] = dict(kw, **autotune.split(cfg))

    def step():
        su = pbng.tip_decompose(dg, "U", P=args.P, with_stats=True, **kws["U"])[1]
        sv = pbng.tip_decompose(dg, "V", P=args.P, with_stats=True, **kws["V"])[1]
        return su, sv

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    # ---- timed region (device time per step; L2 flushed between steps)
    stats = []
    times = []
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats.append(step())
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    ms_max = max_over_ranks(sum(times), ws, dev)
    wedges_step = tip_wedges(stats[0][0]) + tip_wedges(stats[0][1])
    value = whole_job_rate(wedges_step * args.steps, ws, ms_max / 1000.0)

    # ---- kernel roofline: dominant kernel group, CUDA events around every
    # launch of a group.  Graph-captured rounds run the same peel kernels
    # inside a device loop where no per-launch event can be placed, so the
    # roofline then comes from extra steps with host-driven rounds (untimed
    # for the headline value).
    roof_stats = stats
    if args.graph_rounds:
        host_kws = {s: dict(kws[s], graph_rounds=False) for s in kws}
        roof_stats = []
        for _ in range(min(args.steps, 2)):
            flush.zero_()
            roof_stats.append((pbng.tip_decompose(dg, "U", P=args.P, with_stats=True, **host_kws["U"])[1],
                               pbng.tip_decompose(dg, "V", P=args.P, with_stats=True, **host_kws["V"])[1]))
    groups = {"count": ("ns_k_count", "bytes_count", "n_k_count"), "peel": ("ns_k_peel", "bytes_peel", "n_k_peel"),
              "fd": ("ns_k_fd", "bytes_fd", "n_k_fd")}
    agg = {}
    for k, (tn, bn, nn) in groups.items():
        ns = sum(s[tn] for st in roof_stats for s in st)
        by = sum(s[bn] for st in roof_stats for s in st)
        nl = sum(s[nn] for st in roof_stats for s in st)
        agg[k] = (ns, by, nl)
    dom = max(agg, key=lambda k: agg[k][0])
    ns, by, nl = agg[dom]
    peak, peak_kind = peaks()
    achieved = by / ns if ns else 0.0  # bytes per ns == GB/s
    tr = ncu_traffic(dom)
    roofline = {"bound": "hbm", "kernel_group": dom, "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                "unit": "GB/s", "frac": achieved / peak, "traffic": tr,
                "timing": "CUDA events per launch" + (", host-driven rounds (same kernels)" if args.graph_rounds else ""),
                "launches": nl, "ms_per_launch": ns / 1e6 / max(nl, 1),
                "groups": {k: {"ms": v[0] / 1e6, "GB": v[1] / 1e9, "launches": v[2],
                               "GBps": (v[1] / v[0] if v[0] else 0.0)} for k, v in agg.items()}}

    # ---- end to end through the C ABI with host buffers (pinned), copies inside
    pin_off = torch.from_numpy(np.ascontiguousarray(g.u_off).view(np.int64)).pin_memory()
    pin_adj = torch.from_numpy(np.ascontiguousarray(g.u_adj).view(np.int32)).pin_memory()

    class HostG:
        nu, nv = g.nu, g.nv
        u_off = pin_off.numpy().view(np.uint64)
        u_adj = pin_adj.numpy().view(np.uint32)

    hg = HostG()
    e2e_t = []
    e2e_w = 0
    if not args.no_e2e:
        pbng.tip_decompose_host(hg, "U", P=args.P, **kws["U"])
    for _ in range(0 if args.no_e2e else max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, su = pbng.tip_decompose_host(hg, "U", P=args.P, with_stats=True, **kws["U"])
        _, sv = pbng.tip_decompose_host(hg, "V", P=args.P, with_stats=True, **kws["V"])
        e2e_t.append(time.perf_counter() - t0)
        e2e_w += tip_wedges(su) + tip_wedges(sv)
    e2e_max = max_over_ranks(sum(e2e_t), ws, dev)
    e2e_value = whole_job_rate(e2e_w, ws, e2e_max) if e2e_t else None
    h2d = 2 * ((g.nu + 1) * 8 + g.m * 4)
    d2h = (g.nu + g.nv) * 8

    ms_step = ms_max / args.steps
    rec = {}
    if extras:  # the batched / learned comparison of the metric, and the wing workload
        graphs = [x for j in jobs["batch"] for x in j.get()]
        rec["batched"] = record_batched(pbng, graphs, dev, flush)
        del graphs
        rec["learned"] = record_learned(pbng, jobs["learned"].get(), dev, flush)
        rec["wing"] = record_wing(pbng, jobs["wing"].get(), dev, flush)
    pool.close()

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            import platform
            import oracle
            oracle.build()
            w, dt = oracle_sample(SAMPLE)
            cpu = {"value": w / dt, "unit": "wedges/s", "cores": 1, "kind": "oracle", "sample": SAMPLE_DESC,
                   "seconds": dt, "host": platform.machine(),
                   "wedges": "the oracle's own wedge visits (2 sum_y d_y^2 per side, exact for its loops); the GPU "
                             "line counts the wedges its own method visits"}
            full = full_graph_oracle_seconds()
            if full:  # like for like: the same full graph, time per decomposition of both sides
                full["gpu_ms_per_step"] = ms_step
                full["time_ratio"] = full["seconds"] / (ms_step / 1e3)
                cpu["full_graph"] = full
            # the counting step alone, like for like: the oracle's per-vertex
            # counts of the U side of the full graph on every host core against
            # the GPU's counting phase of the U-side decomposition
            t0 = time.perf_counter()
            _, threads = oracle.vertex_counts_parallel(g, "U")
            dt_c = time.perf_counter() - t0
            dvf = np.bincount(g.u_adj, minlength=g.nv).astype(np.float64)
            gpu_count_ms = stats[0][0]["ns_count"] / 1e6
            cpu["count_all_cores"] = {
                "what": "per-vertex butterfly counts of the U side of the full graph (Sec. 2.1 definition, 2-hop "
                        "traversal), oracle on every host thread", "cores": threads, "host": platform.machine(),
                "seconds": dt_c, "wedge_visits": float((dvf ** 2).sum()),
                "value": float((dvf ** 2).sum()) / dt_c, "unit": "wedges/s",
                "gpu_count_phase_ms": gpu_count_ms, "time_ratio": dt_c / (gpu_count_ms / 1e3)}
        s0u, s0v = stats[0]
        line = {
            "metric": "tip decomposition wedges/s (both sides)", "value": value, "unit": "wedges/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic (seeded Chung-Lu generator)",
            "config": {"workload": WORKLOAD_DESC, "name": WORKLOAD, "P": args.P, "sides": "U,V",
                       "graph_rounds": args.graph_rounds, "recount": not args.no_recount, "schedule": tuned,
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "l2": "flushed between steps (256 MB write)", "nu": g.nu, "nv": g.nv, "m": g.m,
                       "wedges_per_step": wedges_step,
                       "rounds_u": s0u["rounds"], "rounds_v": s0v["rounds"], "recounts_u": s0u["recounts"],
                       "recounts_v": s0v["recounts"], "parts_u": s0u["parts_used"], "parts_v": s0v["parts_used"],
                       "phase_ms_u": {k: s0u["ns_" + k] / 1e6 for k in ("setup", "count", "cd", "part", "fd", "total")},
                       "phase_ms_v": {k: s0v["ns_" + k] / 1e6 for k in ("setup", "count", "cd", "part", "fd", "total")}},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "wedges/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": 1000 * sum(e2e_t) / len(e2e_t) if e2e_t else None},
            "gpu_launches": int(sum(s["launches"] for st in stats for s in st)),
            "clocks": clk.summary(),
            **rec,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
