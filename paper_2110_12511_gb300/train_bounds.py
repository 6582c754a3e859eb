"""Train the learned bound proposer and compare it with find_range.

    python -m paper_2110_12511_gb300.train_bounds --graphs 40 --out DIR

Training graphs: Chung-Lu bipartite graphs seeded 5000 + t with edge counts
log-uniform in [m_lo, m_hi], exponent uniform in [2.0, 2.8] (both sides),
|U|:|V| uniform in [1, 8], |U| + |V| = m / 10, degree cap 50k.  Targets come
from exact decompositions (see learned.py).  Evaluation: the 5M x 1M,
60M-edge Chung-Lu graph (exponents 2.1 / 2.3), tip of U with P = 200,
learned bounds against find_range, identical tip numbers required.
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
        th, st = pbng.tip_decompose(dg, "U", P=P, with_stats=True, mlp=params if mode == "learned" else None)
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=40)
    ap.add_argument("--m-lo", type=int, default=500000)
    ap.add_argument("--m-hi", type=int, default=20000000)
    ap.add_argument("--P", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_2110_12511_gb300", "data"))
    ap.add_argument("--no-eval", action="store_true")
    ap.add_argument("--heldout", type=int, default=6)
    args = ap.parse_args()
    from paper_2110_12511_gb300 import build as b
    b.build()
    import torch
    from paper_2110_12511_gb300 import learned
    torch.cuda.set_device(0)
    X, T, info = [], [], []
    t0 = time.time()
    for t in range(args.graphs):
        g = training_graph(t, args.m_lo, args.m_hi)
        f, y, inf = learned.training_example(g, "U", args.P)
        X.append(f)
        T.append(y)
        info.append({"graph": t, "m": g.m, **inf})
        print(json.dumps(info[-1]), flush=True)
    gen_s = time.time() - t0
    X, T = np.stack(X), np.stack(T)
    params, losses = learned.train(X, T, args.P - 1, epochs=args.epochs)
    path = os.path.join(args.out, f"bound_mlp_p{args.P}.npz")
    learned.save(path, params.cpu().numpy(), args.P - 1, {"graphs": args.graphs, "m": [args.m_lo, args.m_hi]})
    summary = {"train_graphs": args.graphs, "data_s": gen_s, "loss_first": losses[0], "loss_last": losses[-1],
               "winners": {w: sum(1 for i in info if i["winner"] == w) for w in {i["winner"] for i in info}}}
    if not args.no_eval:
        mlp = (params, learned.HID, args.P - 1)
        held = []
        for t in range(1000, 1000 + args.heldout):  # same distribution, seeds never trained on
            r = evaluate(mlp, P=args.P, g=training_graph(t, args.m_lo, args.m_hi))
            held.append({"graph": t, "speedup": r["speedup"], "estimator_s": r["estimator"]["best_s"],
                         "learned_s": r["learned"]["best_s"]})
        summary["heldout"] = held
        summary["heldout_geomean_speedup"] = float(np.exp(np.mean([np.log(h["speedup"]) for h in held])))
        summary["eval_chunglu_5m_1m_60m"] = evaluate(mlp, P=args.P)
    print(json.dumps(summary), flush=True)
    with open(os.path.join(args.out, f"bound_mlp_p{args.P}_summary.json"), "w") as f:
        json.dump({"summary": summary, "examples": info}, f, indent=1)


if __name__ == "__main__":
    main()
