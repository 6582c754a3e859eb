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
