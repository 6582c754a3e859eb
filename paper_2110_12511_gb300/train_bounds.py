"""Train the learned bound proposers and compare them with find_range.

    python -m paper_2110_12511_gb300.train_bounds [--kind tip|wing] [--graphs N] [--out DIR]

Tip: Chung-Lu bipartite graphs seeded 5000 + t with edge counts log-uniform
in [m_lo, m_hi] (default 1M-60M), exponent uniform in [2.0, 2.8] (both
sides), |U|:|V| uniform in [1, 8], |U| + |V| = m / 10, degree cap 50k.
Evaluation: the 5M x 1M, 60M-edge Chung-Lu graph (exponents 2.1 / 2.3), tip
of U with P = 200, learned bounds against find_range, identical tip numbers
required, plus held-out graphs of the training distribution (seeds 1000+).

Wing: the planted recipe of the 500k x 100k workload at other sizes (seeded
7000 + t, base edges log-uniform in [0.5M, 5M], |U| = m / 10, |V| = m / 50,
exponents uniform in [2.1, 2.5], 0-200 planted bicliques of 20-200 x
20-200), P = 100; evaluation on the planted 500k x 100k graph.

Targets come from exact decompositions (see learned.py).  The graphs are
generated by a pool of host processes (started before the first GPU call)
while the GPU times the previous ones.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def training_graph(t, m_lo, m_hi):
    import bigraph_gen as gen
    rng = np.random.default_rng(5000 + t)
    m = int(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi))))
    g = float(rng.uniform(2.0, 2.8))
    r = float(rng.uniform(1.0, 8.0))
    n = m // 10
    nu = max(int(n * r / (1 + r)), 2)
    nv = max(n - nu, 2)
    return gen.chung_lu(nu, nv, m, g, g, 50000, seed=5000 + t)


def training_wing_graph(t, m_lo, m_hi):
    """Chung-Lu graph with planted bicliques (the recipe of the planted
    500k x 100k workload at other sizes)."""
    import bigraph_gen as gen
    rng = np.random.default_rng(7000 + t)
    m = int(np.exp(rng.uniform(np.log(m_lo), np.log(m_hi))))
    gu = float(rng.uniform(2.1, 2.5))
    gv = float(rng.uniform(2.1, 2.5))
    nplant = int(rng.integers(0, 201))
    return gen.make(dict(kind="chung_lu", nu=max(m // 10, 2), nv=max(m // 50, 2), m=m, gu=gu, gv=gv, dmax=50000,
                         seed=7000 + t, nplant=nplant, plant_lo=20, plant_hi=200))


def _graph_job(job):
    t, m_lo, m_hi, kind = job
    return (training_wing_graph if kind == "wing" else training_graph)(t, m_lo, m_hi)


def _pool(workers):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(workers)


def evaluate(params, P=200, reps=2, g=None):
    """Learned bounds against find_range on one graph (default: the 60M-edge one)."""
    import torch
    import bigraph_gen as gen
    import paper_2110_12511_gb300 as pbng
    g = g if g is not None else gen.make("chunglu_5m_1m_60m")
    dg = pbng.to_device(g)
    res = {}
    ref = None
    for mode in ("estimator", "learned", "estimator", "learned"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        th, st = pbng.tip_decompose(dg, "U", P=P, with_stats=True, graph_rounds=True,
                                    mlp=params if mode == "learned" else None)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        th = pbng.as_u64(th)
        if ref is None:
            ref = th
        assert np.array_equal(th, ref), "learned bounds changed the tip numbers"
        r = res.setdefault(mode, {"s": []})
        r["s"].append(dt)
        r.update({k: st[k] for k in ("rounds", "parts_used", "launches", "ns_cd", "ns_fd", "fd_work_max", "fd_work_sum",
                                      "wedges_cd")})
    for r in res.values():
        r["best_s"] = min(r["s"])
        r["fd_imbalance"] = r["fd_work_max"] / max(1.0, r["fd_work_sum"] / max(1, r["parts_used"]))
    res["speedup"] = res["estimator"]["best_s"] / res["learned"]["best_s"]
    return res


def evaluate_wing(params, P=100, g=None):
    """Learned wing bounds against find_range (default: the planted 500k x 100k graph)."""
    import torch
    import bigraph_gen as gen
    import paper_2110_12511_gb300 as pbng
    g = g if g is not None else gen.make("chunglu_500k_100k_5m_planted")
    dg = pbng.to_device(g)
    res, ref = {}, None
    for mode in ("estimator", "learned", "estimator", "learned"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        th, st = pbng.wing_decompose(dg, P=P, with_stats=True, mlp=params if mode == "learned" else None)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        th = pbng.as_u64(th)
        if ref is None:
            ref = th
        assert np.array_equal(th, ref), "learned bounds changed the wing numbers"
        r = res.setdefault(mode, {"s": []})
        r["s"].append(dt)
        r.update({k: st[k] for k in ("rounds", "parts_used", "ns_cd", "ns_fd", "fd_work_max", "fd_work_sum")})
    for r in res.values():
        r["best_s"] = min(r["s"])
    res["speedup"] = res["estimator"]["best_s"] / res["learned"]["best_s"]
    return res


def run(args, kind):
    from paper_2110_12511_gb300 import build as b
    pool = _pool(args.workers)  # before any GPU call
    jobs = pool.imap(_graph_job, [(t, args.m_lo, args.m_hi, kind) for t in range(args.graphs)])
    b.build()
    import torch
    from paper_2110_12511_gb300 import learned
    torch.cuda.set_device(0)
    X, T, info = [], [], []
    t0 = time.time()
    for t in range(args.graphs):
        g = next(jobs)
        if kind == "wing":
            f, y, inf = learned.wing_training_example(g, args.P)
        else:
            f, y, inf = learned.training_example(g, "U", args.P)
        X.append(f)
        T.append(y)
        info.append({"graph": t, "m": g.m, **inf})
        print(json.dumps(info[-1]), flush=True)
    gen_s = time.time() - t0
    held_graphs = pool.map(_graph_job, [(t, args.m_lo, args.m_hi, kind) for t in range(1000, 1000 + args.heldout)])
    pool.close()
    X, T = np.stack(X), np.stack(T)
    params, losses = learned.train(X, T, args.P - 1, epochs=args.epochs)
    stem = f"bound_mlp_wing_p{args.P}" if kind == "wing" else f"bound_mlp_p{args.P}"
    learned.save(os.path.join(args.out, stem + ".npz"), params.cpu().numpy(), args.P - 1,
                 {"kind": kind, "graphs": args.graphs, "m": [args.m_lo, args.m_hi]})
    summary = {"kind": kind, "train_graphs": args.graphs, "m": [args.m_lo, args.m_hi], "data_s": gen_s,
               "loss_first": losses[0], "loss_last": losses[-1],
               "winners": {w: sum(1 for i in info if i["winner"] == w) for w in {i["winner"] for i in info}}}
    if not args.no_eval:
        mlp = (params, learned.HID, args.P - 1)
        ev = evaluate_wing if kind == "wing" else evaluate
        held = []
        for t, g in zip(range(1000, 1000 + args.heldout), held_graphs):  # same distribution, never trained on
            r = ev(mlp, P=args.P, g=g)
            held.append({"graph": t, "m": g.m, "speedup": r["speedup"], "estimator_s": r["estimator"]["best_s"],
                         "learned_s": r["learned"]["best_s"]})
        summary["heldout"] = held
        summary["heldout_geomean_speedup"] = float(np.exp(np.mean([np.log(h["speedup"]) for h in held])))
        key = "eval_chunglu_500k_100k_5m_planted" if kind == "wing" else "eval_chunglu_5m_1m_60m"
        summary[key] = ev(mlp, P=args.P)
    print(json.dumps(summary), flush=True)
    with open(os.path.join(args.out, stem + "_summary.json"), "w") as f:
        json.dump({"summary": summary, "examples": info}, f, indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", default="tip", choices=["tip", "wing"])
    ap.add_argument("--graphs", type=int, default=None, help="default: 160 (tip), 40 (wing)")
    ap.add_argument("--m-lo", type=int, default=None, help="default: 1M (tip), 0.5M (wing)")
    ap.add_argument("--m-hi", type=int, default=None, help="default: 60M (tip), 5M (wing)")
    ap.add_argument("--P", type=int, default=None, help="default: 200 (tip), 100 (wing)")
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--workers", type=int, default=max(1, min(8, (os.cpu_count() or 2) - 2)))
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_2110_12511_gb300", "data"))
    ap.add_argument("--no-eval", action="store_true")
    ap.add_argument("--heldout", type=int, default=6)
    args = ap.parse_args()
    wing = args.kind == "wing"
    for k, tip_v, wing_v in (("graphs", 160, 40), ("m_lo", 1000000, 500000), ("m_hi", 60000000, 5000000),
                             ("P", 200, 100)):
        if getattr(args, k) is None:
            setattr(args, k, wing_v if wing else tip_v)
    os.makedirs(args.out, exist_ok=True)
    run(args, args.kind)


if __name__ == "__main__":
    main()
