"""Write full-size expected results computed by the CPU oracle.

For each full-size workload this records a hash of the generated graph (so a
drift in the generator is detected), then runs the oracle's bottom-up peeling
(Alg. 2) and stores a SHA-256 of the resulting uint64 tip numbers together
with summary values and a fixed sample of (index, value) pairs.  Only
``oracle`` and ``bigraph_gen`` are used.  Run once (the tip jobs take tens
of minutes of CPU time, the full-size wing job hours); the GPU tests compare against the stored files.

    python tests/golden/make_golden.py [name ...]
"""
from __future__ import annotations

import hashlib
import json
import multiprocessing as mp
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

JOBS = {
    # name: (workload, side) ; batch jobs enumerate the 4,096 batch graphs
    "tip_chunglu_1m_200k_20m_U": ("chunglu_1m_200k_20m", "U"),
    "tip_chunglu_1m_200k_20m_V": ("chunglu_1m_200k_20m", "V"),
    "tip_chunglu_5m_1m_60m_U": ("chunglu_5m_1m_60m", "U"),
    "tip_batch_4096_U": ("batch", "U"),
    # wing numbers (side "E": every edge) of the planted 500k x 100k graph,
    # and of the same recipe on a 1M-edge Chung-Lu base with all 200 planted
    # bicliques kept
    "wing_chunglu_500k_100k_5m_planted": ("chunglu_500k_100k_5m_planted", "E"),
    "wing_chunglu_500k_100k_1m_planted": ("chunglu_500k_100k_1m_planted", "E"),
}
BATCH_N, BATCH_SEED0 = 4096, 1000


def graph_sha(g) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.u_off, dtype=np.uint64).tobytes())
    h.update(np.ascontiguousarray(g.u_adj, dtype=np.uint32).tobytes())
    return h.hexdigest()


def samples(theta: np.ndarray, k: int = 64):
    rng = np.random.default_rng(20211024)
    idx = np.unique(np.concatenate([rng.integers(0, theta.size, size=k), [int(np.argmax(theta))]]))
    return [[int(i), int(theta[i])] for i in idx]


def run(name: str) -> dict:
    import bigraph_gen as gen
    import oracle
    workload, side = JOBS[name]
    t0 = time.time()
    if workload == "batch":
        h = hashlib.sha256()
        gh = hashlib.sha256()
        thetas = []
        for i in range(BATCH_N):
            g = gen.batch_graph(BATCH_SEED0 + i)
            gh.update(graph_sha(g).encode())
            th = oracle.tip(g, side).astype(np.uint64)
            h.update(th.tobytes())
            thetas.append(th)
        allt = np.concatenate(thetas)
        rec = {"graph_sha256": gh.hexdigest(), "theta_sha256": h.hexdigest(), "n": int(allt.size),
               "max": int(allt.max()), "sum": int(allt.sum(dtype=np.uint64)),
               "per_graph_sha256": [hashlib.sha256(t.tobytes()).hexdigest()[:16] for t in thetas]}
    else:
        g = gen.make(workload)
        th = (oracle.wing(g) if side == "E" else oracle.tip(g, side)).astype(np.uint64)
        rec = {"graph_sha256": graph_sha(g), "theta_sha256": hashlib.sha256(th.tobytes()).hexdigest(),
               "n": int(th.size), "max": int(th.max()), "sum": int(th.sum(dtype=np.uint64)), "samples": samples(th)}
    rec.update({"job": name, "workload": workload, "side": side, "oracle": "bottom-up peeling (Alg. 2), oracle/oracle.c", "host_cores_used": 1,
                "host": platform.machine(),
                "cpu_seconds": round(time.time() - t0, 1)})
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(rec, f, indent=1)
    return rec


if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(names), os.cpu_count() or 1)) as pool:
        for rec in pool.imap_unordered(run, names):
            print(rec["job"], rec["theta_sha256"][:16], rec["cpu_seconds"], "s", flush=True)
