"""Brute-force definitions used to pin the oracle (tiny graphs only).

Each routine restates a definition from the paper directly, with no peeling
order, no clamp and no shared code with ``oracle/``:

* butterflies by 4-tuple enumeration (a butterfly is a 2,2-biclique, Sec. 2);
* tip / wing numbers as "the largest k such that the entity lies in a
  subgraph whose members all have >= k butterflies inside it" (Def. 1-2,
  Sec. 2.2), either by enumerating every subset or by the k-level fixed point
  (remove members with < k butterflies until none is left to remove).
"""
from __future__ import annotations

from itertools import combinations

import numpy as np


def adjacency(g):
    a = np.zeros((g.nu, g.nv), dtype=np.int64)
    eu, ev = g.edges()
    a[eu.astype(np.int64), ev.astype(np.int64)] = 1
    return a


def edge_index(g):
    eu, ev = g.edges()
    return {(int(u), int(v)): i for i, (u, v) in enumerate(zip(eu, ev))}


def butterflies(g):
    """All butterflies as tuples (u1, u2, v1, v2) with u1<u2, v1<v2."""
    a = adjacency(g)
    out = []
    for u1, u2 in combinations(range(g.nu), 2):
        common = np.nonzero(a[u1] & a[u2])[0]
        for v1, v2 in combinations(common.tolist(), 2):
            out.append((u1, u2, v1, v2))
    return out


def counts_by_enumeration(g):
    """(per-U-vertex, per-V-vertex, per-edge, total) butterfly counts."""
    eidx = edge_index(g)
    cu = np.zeros(g.nu, dtype=np.int64)
    cv = np.zeros(g.nv, dtype=np.int64)
    ce = np.zeros(g.m, dtype=np.int64)
    bs = butterflies(g)
    for (u1, u2, v1, v2) in bs:
        cu[[u1, u2]] += 1
        cv[[v1, v2]] += 1
        for e in ((u1, v1), (u1, v2), (u2, v1), (u2, v2)):
            ce[eidx[e]] += 1
    return cu, cv, ce, len(bs)


def pair_butterflies(g):
    """B[u, u'] = C(|N_u cap N_u'|, 2), zero diagonal (common neighbours by A A^T)."""
    a = adjacency(g)
    c = a @ a.T
    b = c * (c - 1) // 2
    np.fill_diagonal(b, 0)
    return b


def tip_by_subsets(g):
    """Tip numbers of U: max over subsets S containing u of min_{w in S} sup_w(S)."""
    b = pair_butterflies(g)
    n = g.nu
    best = np.zeros(n, dtype=np.int64)
    for mask in range(1, 1 << n):
        members = [i for i in range(n) if mask >> i & 1]
        sub = b[np.ix_(members, members)]
        k = int(sub.sum(axis=1).min())
        for i in members:
            if k > best[i]:
                best[i] = k
    return best


def tip_by_fixpoint(g):
    """Tip numbers of U: theta_u = max k with u in the k-level, where the
    k-level is what remains after repeatedly removing members with < k
    butterflies among the remaining members."""
    b = pair_butterflies(g)
    n = g.nu
    theta = np.zeros(n, dtype=np.int64)
    k = 1
    alive = np.ones(n, dtype=bool)
    while alive.any():
        while True:
            sup = b[:, alive].sum(axis=1)
            drop = alive & (sup < k)
            if not drop.any():
                break
            alive &= ~drop
        theta[alive] = k
        k += 1
    return theta


def _edge_butterflies(g):
    eidx = edge_index(g)
    return [tuple(eidx[e] for e in ((u1, v1), (u1, v2), (u2, v1), (u2, v2)))
            for (u1, u2, v1, v2) in butterflies(g)]


def wing_by_subsets(g):
    """Wing numbers: max over edge subsets S containing e of the minimum
    number of butterflies (all 4 edges in S) an edge of S lies in."""
    m = g.m
    bmask = [sum(1 << e for e in bf) for bf in _edge_butterflies(g)]
    best = [0] * m
    for mask in range(1, 1 << m):
        inside = [bm for bm in bmask if bm & mask == bm]
        sup = [0] * m
        for bm in inside:
            for e in range(m):
                if bm >> e & 1:
                    sup[e] += 1
        members = [e for e in range(m) if mask >> e & 1]
        k = min(sup[e] for e in members)
        for e in members:
            if k > best[e]:
                best[e] = k
    return np.array(best, dtype=np.int64)


def wing_by_fixpoint(g):
    """Wing numbers by the k-level fixed point over edges."""
    bfs = np.array(_edge_butterflies(g), dtype=np.int64).reshape(-1, 4)
    m = g.m
    theta = np.zeros(m, dtype=np.int64)
    alive = np.ones(m, dtype=bool)
    k = 1
    while alive.any():
        while True:
            live_b = alive[bfs].all(axis=1) if len(bfs) else np.zeros(0, dtype=bool)
            sup = np.bincount(bfs[live_b].ravel(), minlength=m) if len(bfs) else np.zeros(m, dtype=np.int64)
            drop = alive & (sup < k)
            if not drop.any():
                break
            alive &= ~drop
        theta[alive] = k
        k += 1
    return theta
