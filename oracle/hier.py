"""Oracle of k-tip retrieval (TEST INFRASTRUCTURE ONLY: only tests/ use it).

Def. 2: a k-tip of side X is a maximal set of vertices, each in at least k
butterflies of the subgraph induced on (that set, Y), any two connected by a
series of butterflies.  Tip numbers index the hierarchy (Sec. 2.2): the
k-tips are the butterfly-connected components of X_k = {x : theta_x >= k}.
Two vertices of X_k share a butterfly exactly when they have at least two
common neighbours, so this oracle takes the common-neighbour counts of X_k
as the sparse product A_k A_k^T (a library matmul), keeps the pairs with a
count of 2 or more, and labels connected components (a library routine),
each by its smallest member; vertices below k get 0xffffffff.
"""
from __future__ import annotations

import numpy as np

NONE = 0xFFFFFFFF


def tip_components(g, side, theta, k):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    h = g if side == "U" else g.swapped()
    nx, ny = h.nu, h.nv
    theta = np.asarray(theta, dtype=np.uint64)
    mem = theta >= np.uint64(k)
    out = np.full(nx, NONE, dtype=np.uint32)
    ids = np.nonzero(mem)[0]
    if ids.size == 0:
        return out
    off = np.asarray(h.u_off, dtype=np.int64)
    adj = np.asarray(h.u_adj, dtype=np.int64)
    A = csr_matrix((np.ones(adj.size, dtype=np.int64), adj, off), shape=(nx, ny))
    Ak = A[ids]
    C = (Ak @ Ak.T).tocoo()
    keep = (C.row != C.col) & (C.data >= 2)
    E = csr_matrix((np.ones(int(keep.sum()), dtype=np.int8), (C.row[keep], C.col[keep])), shape=(ids.size, ids.size))
    ncomp, lab = connected_components(E, directed=False)
    smallest = np.full(ncomp, np.iinfo(np.int64).max, dtype=np.int64)
    np.minimum.at(smallest, lab, ids)
    out[ids] = smallest[lab].astype(np.uint32)
    return out


def wing_components(g, theta, k):
    """k-wings (Def. 1) from wing numbers, U-CSR edge order.  E_k = edges with
    theta >= k; for every vertex pair (u, u') the common neighbours v with
    (u, v) and (u', v) both in E_k are listed; a pair with two or more of them
    forms butterflies inside E_k that hold all of those edges, so they are
    joined (union-find); each component is labelled by its smallest edge id."""
    theta = np.asarray(theta, dtype=np.uint64)
    m = int(g.m)
    out = np.full(m, NONE, dtype=np.uint32)
    mem = theta >= np.uint64(k)
    off = np.asarray(g.u_off, dtype=np.int64)
    adj = np.asarray(g.u_adj, dtype=np.int64)
    vl = [[] for _ in range(g.nv)]  # v -> [(u, e)] over E_k
    for u in range(g.nu):
        for e in range(off[u], off[u + 1]):
            if mem[e]:
                vl[adj[e]].append((u, e))
    par = list(range(m))

    def find(x):
        while par[x] != x:
            par[x] = par[par[x]]
            x = par[x]
        return x

    def unite(a, b):
        a, b = find(a), find(b)
        if a != b:
            par[max(a, b)] = min(a, b)

    for u in range(g.nu):
        pairs = {}
        for e in range(off[u], off[u + 1]):
            if not mem[e]:
                continue
            for u2, e2 in vl[adj[e]]:
                if u2 > u:
                    pairs.setdefault(u2, []).append((e, e2))
        for lst in pairs.values():
            if len(lst) >= 2:
                r = lst[0][0]
                for e, e2 in lst:
                    unite(e, r)
                    unite(e2, r)
    for e in range(m):
        if mem[e]:
            out[e] = find(e)
    return out
