"""Learned coarse-phase bounds (the batched/learned configuration).

A 3-layer MLP (FP32, width 128) maps the 128 histogram features of a graph
(``pbng_bound_features``: half-octave degree histogram of the peeled side and
histogram of how far below the largest initial butterfly count K each count's
bit length is) to upper bounds theta(2) < theta(3) < ... of the coarse-phase
ranges, encoded relative to K as y_i = log2(1 + b_i) / log2(1 + K).  Forward, backward and Adam steps run in the
library's own CUDA kernels (``pbng_mlp_*``); this module only orchestrates.

Training targets come from the method itself: for each training graph the
exact tip numbers are computed, a few candidate bound sequences are built
(the find_range estimator's own bounds, work quantiles of the exact numbers
and blends of the two in log space), each is timed on the GPU, and the
fastest becomes the target.  Any bounds give identical tip numbers (Sec. 4.1,
Th. 2), so the network can only change speed; a bound that would peel nothing
falls back to find_range inside the library.

The wing proposer is the same network over the edges
(``pbng_wing_bound_features``: min(d_u, d_v) per edge and the per-edge
initial butterfly counts), with work quantiles taken over the exact wing
numbers weighted by support, the wing work proxy (Sec. 3.3.2).
"""
from __future__ import annotations

import os
import time

import numpy as np

from . import (BOUNDS_ESTIMATOR, as_u64, bound_features, mlp_adam, mlp_grad, tip_decompose, to_device,
               wing_bound_features, wing_decompose)

NIN, HID = 128, 128
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "bound_mlp_p200.npz")
WING_WEIGHTS = os.path.join(HERE, "data", "bound_mlp_wing_p100.npz")
BLENDS = (0.25, 0.5, 0.75)


def n_params(nin=NIN, hid=HID, out=199):
    return nin * hid + hid + hid * hid + hid + hid * out + out


def init_params(out, seed=0, nin=NIN, hid=HID):
    """He-initialised weights, zero biases (float32, packed layout of pbng_mlp_forward)."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, np.sqrt(2.0 / nin), size=nin * hid), np.zeros(hid),
             rng.normal(0, np.sqrt(2.0 / hid), size=hid * hid), np.zeros(hid),
             rng.normal(0, np.sqrt(1.0 / hid), size=hid * out), np.full(out, 0.3)]
    return np.concatenate(parts).astype(np.float32)


def encode(bounds, out, K):
    """Targets y_i = log2(1 + b_i) / log2(1 + K), padded to `out` with the last value."""
    b = np.asarray(bounds, dtype=np.float64)
    y = np.log2(1.0 + b) / np.log2(1.0 + max(float(K), 1.0)) if b.size else np.zeros(1)
    if y.size < out:
        y = np.concatenate([y, np.full(out - y.size, y[-1])])
    return y[:out].astype(np.float32)


def decode(y, K):
    """Strictly increasing integer bounds from network outputs (as the library does)."""
    out = []
    for v in np.asarray(y, dtype=np.float64):
        e = min(max(v * np.log2(1.0 + float(K)), 0.0), 63.0)
        b = max(int(round(2.0 ** e)) - 1, 1)
        if out and b <= out[-1]:
            continue
        out.append(b)
    return np.array(out, dtype=np.uint64)


def quantile_bounds(theta, work, P):
    """Upper bounds splitting the total work into P equal parts along theta."""
    o = np.argsort(theta, kind="stable")
    th, cw = theta[o], np.cumsum(work[o].astype(np.float64))
    out = []
    for i in range(1, P):
        k = min(int(np.searchsorted(cw, cw[-1] * i / P)), th.size - 1)
        b = int(th[k]) + 1
        if not out or b > out[-1]:
            out.append(b)
    return np.array(out, dtype=np.uint64)


def blend(a, b, t, P):
    """Log-space blend of two bound sequences resampled to P-1 points."""
    def res(x):
        x = np.log2(1.0 + np.asarray(x, dtype=np.float64))
        if x.size == 0:
            return np.zeros(P - 1)
        return np.interp(np.linspace(0, 1, P - 1), np.linspace(0, 1, x.size), x)
    y = (1 - t) * res(a) + t * res(b)
    out = []
    for v in y:
        bb = max(int(round(2.0 ** v)) - 1, 1)
        if not out or bb > out[-1]:
            out.append(bb)
    return np.array(out, dtype=np.uint64)


def _fastest(run, cands, reps):
    """Name of the fastest candidate: run(bounds or None) timed on the GPU."""
    import torch
    times = {}
    for name, b in cands.items():
        best = 1e30
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run(b if name != "estimator" else None)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        times[name] = best
    return min(times, key=times.get), times


def candidates(est, wq, P):
    c = {"estimator": est, "work_quantiles": wq}
    for t in BLENDS:
        c[f"blend_{t}"] = blend(est, wq, t, P)
    return c


def training_example(g, side, P, reps=2, graph_rounds=True):
    """(features, target y, info) for one graph: the fastest candidate bounds
    (timed as the decomposition runs by default: graph-captured rounds)."""
    import torch
    from . import count
    dg = to_device(g)
    feat = bound_features(dg, side).cpu().numpy()
    cu, cv, _ = count(dg, vertices=True)
    K = int(as_u64(cu if side == "U" else cv).max()) if (g.nu if side == "U" else g.nv) else 0
    used = np.zeros(P, dtype=np.uint64)
    theta, st = tip_decompose(dg, side, P=P, with_stats=True, bounds_out=used)
    est = used[:max(st["parts_used"] - 1, 0)].copy()
    theta = as_u64(theta).astype(np.float64)
    h = g if side == "U" else g.swapped()
    dh = np.diff(h.u_off).astype(np.int64)
    do = np.bincount(h.u_adj, minlength=h.nv).astype(np.float64)
    w = np.bincount(np.repeat(np.arange(h.nu), dh), weights=do[h.u_adj], minlength=h.nu)
    wq = quantile_bounds(theta, w, P)
    cands = candidates(est, wq, P)
    win, times = _fastest(lambda b: tip_decompose(dg, side, P=P, bounds=b, graph_rounds=graph_rounds), cands, reps)
    return feat, encode(cands[win], P - 1, K), {"times": times, "winner": win, "K": K}


def wing_training_example(g, P, reps=2):
    """(features, target y, info) for the wing proposer on one graph."""
    from . import count
    dg = to_device(g)
    feat = wing_bound_features(dg).cpu().numpy()
    _, _, ce = count(dg, vertices=False, edges=True)
    sup = as_u64(ce).astype(np.float64)
    K = int(sup.max()) if sup.size else 0
    used = np.zeros(P, dtype=np.uint64)
    theta, st = wing_decompose(dg, P=P, with_stats=True, bounds_out=used)
    est = used[:max(st["parts_used"] - 1, 0)].copy()
    wq = quantile_bounds(as_u64(theta).astype(np.float64), sup, P)
    cands = candidates(est, wq, P)
    win, times = _fastest(lambda b: wing_decompose(dg, P=P, bounds=b), cands, reps)
    return feat, encode(cands[win], P - 1, K), {"times": times, "winner": win, "K": K}


def train(X, T, out, epochs=3000, lr=2e-3, seed=0, batch=None, log_every=0):
    """Train the MLP on device with the library's kernels; returns (params, losses)."""
    import torch
    dev = "cuda"
    Xd = torch.as_tensor(np.asarray(X, dtype=np.float32), device=dev).contiguous()
    Td = torch.as_tensor(np.asarray(T, dtype=np.float32), device=dev).contiguous()
    p = torch.as_tensor(init_params(out, seed), device=dev).contiguous()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    dims = (NIN, HID, out)
    losses = []
    n = Xd.shape[0]
    rng = np.random.default_rng(seed)
    for step in range(1, epochs + 1):
        if batch and batch < n:
            idx = torch.as_tensor(rng.choice(n, size=batch, replace=False), device=dev)
            g, loss = mlp_grad(p, dims, Xd[idx].contiguous(), Td[idx].contiguous())
        else:
            g, loss = mlp_grad(p, dims, Xd, Td)
        mlp_adam(p, g, m, v, lr, step)
        losses.append(loss)
        if log_every and step % log_every == 0:
            print(f"step {step} loss {loss:.3e}", flush=True)
    return p, losses


def save(path, params, out, meta=None):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params=np.asarray(params, dtype=np.float32), nin=NIN, hidden=HID, out=out,
             meta=np.array(repr(meta or {})))


def load(path=DEFAULT_WEIGHTS, device="cuda"):
    """(params tensor on device, hidden, out) ready for tip_decompose(mlp=...)
    (or wing_decompose(mlp=...) with WING_WEIGHTS)."""
    import torch
    d = np.load(path)
    return torch.as_tensor(d["params"], device=device).contiguous(), int(d["hidden"]), int(d["out"])
