"""Pins of the k-tip oracle: brute-force butterfly enumeration on tiny graphs
(Def. 2 read directly), complete bipartite graphs, the worked graph G' and
the nesting of the hierarchy."""
import itertools

import numpy as np
import pytest

import bigraph_gen as gen
import oracle
from oracle import hier

pytest.importorskip("scipy")


def brute_components(g, theta, k):
    """Union the U vertices of every butterfly (u1, u2, v1, v2) of the subgraph
    induced on {u : theta_u >= k} and all of V; label by smallest member."""
    off = np.asarray(g.u_off, dtype=np.int64)
    nbr = [set(int(v) for v in g.u_adj[off[u]:off[u + 1]]) for u in range(g.nu)]
    mem = [u for u in range(g.nu) if int(theta[u]) >= k]
    par = {u: u for u in mem}

    def find(u):
        while par[u] != u:
            u = par[u]
        return u

    for u1, u2 in itertools.combinations(mem, 2):
        for v1, v2 in itertools.combinations(range(g.nv), 2):
            if {v1, v2} <= nbr[u1] and {v1, v2} <= nbr[u2]:
                a, b = find(u1), find(u2)
                if a != b:
                    par[max(a, b)] = min(a, b)
    out = np.full(g.nu, hier.NONE, dtype=np.uint32)
    for u in mem:
        out[u] = find(u)
    return out


def rand_graph(nu, nv, p, seed):
    rng = np.random.default_rng(seed)
    eu, ev = np.nonzero(rng.random((nu, nv)) < p)
    return gen.from_edges(nu, nv, eu, ev)


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_tiny(seed):
    g = rand_graph(9, 7, 0.45, seed)
    theta = oracle.tip(g, "U")
    for k in sorted(set(int(t) for t in theta)) + [0, int(theta.max()) + 1]:
        assert np.array_equal(hier.tip_components(g, "U", theta, k), brute_components(g, theta, k)), k


def test_complete_bipartite_is_one_tip():
    a, b = 6, 4
    g = gen.complete(a, b)
    theta = oracle.tip(g, "U")
    assert (theta == (a - 1) * (b * (b - 1) // 2)).all()
    comp = hier.tip_components(g, "U", theta, int(theta[0]))
    assert (comp == 0).all()
    assert (hier.tip_components(g, "U", theta, int(theta[0]) + 1) == hier.NONE).all()


def test_two_disjoint_bicliques_are_two_tips():
    # K_{3,3} on U {0,1,2} x V {0,1,2} and K_{3,3} on U {3,4,5} x V {3,4,5}
    eu = [u for u in range(3) for _ in range(3)] + [u for u in range(3, 6) for _ in range(3)]
    ev = [v for _ in range(3) for v in range(3)] + [v for _ in range(3) for v in range(3, 6)]
    g = gen.from_edges(6, 6, eu, ev)
    theta = oracle.tip(g, "U")
    comp = hier.tip_components(g, "U", theta, 1)
    assert list(comp) == [0, 0, 0, 3, 3, 3]


def test_hierarchy_nests_and_members_are_never_alone():
    g = gen.make("chunglu_5k_1k_50k_planted")
    theta = oracle.tip(g, "U")
    levels = np.unique(theta)
    ks = [int(x) for x in levels[:: max(1, len(levels) // 8)]]
    prev = None
    for k in ks:
        comp = hier.tip_components(g, "U", theta, k)
        mem = comp != hier.NONE
        assert np.array_equal(mem, theta >= k)
        if k >= 1:  # a member has at least k butterflies inside its tip, so a partner
            sizes = np.bincount(comp[mem])
            assert (sizes[comp[mem]] >= 2).all()
        if prev is not None:  # a (higher) k-tip lies inside one lower tip
            pk, pcomp = prev
            for c in np.unique(comp[mem]):
                assert len(np.unique(pcomp[comp == c])) == 1
        prev = (k, comp)


def brute_wing_components(g, theta, k):
    """Union the four edges of every butterfly whose edges all have wing number >= k."""
    off = np.asarray(g.u_off, dtype=np.int64)
    eid = {}
    for u in range(g.nu):
        for e in range(off[u], off[u + 1]):
            eid[(u, int(g.u_adj[e]))] = e
    mem = {e for e in range(g.m) if int(theta[e]) >= k}
    par = {e: e for e in mem}

    def find(x):
        while par[x] != x:
            x = par[x]
        return x

    for u1, u2 in itertools.combinations(range(g.nu), 2):
        for v1, v2 in itertools.combinations(range(g.nv), 2):
            es = [eid.get((u1, v1)), eid.get((u1, v2)), eid.get((u2, v1)), eid.get((u2, v2))]
            if all(e is not None and e in mem for e in es):
                r = min(find(e) for e in es)
                for e in es:
                    par[find(e)] = r
    out = np.full(g.m, hier.NONE, dtype=np.uint32)
    for e in mem:
        out[e] = find(e)
    return out


@pytest.mark.parametrize("seed", range(10))
def test_wing_brute_force_tiny(seed):
    g = rand_graph(8, 7, 0.5, 100 + seed)
    theta = oracle.wing(g)
    for k in sorted(set(int(t) for t in theta)) + [0, int(theta.max()) + 1]:
        assert np.array_equal(hier.wing_components(g, theta, k), brute_wing_components(g, theta, k)), k


def test_wing_complete_and_disjoint_bicliques():
    g = gen.complete(5, 4)
    theta = oracle.wing(g)
    assert (theta == 4 * 3).all()  # (a - 1)(b - 1)
    assert (hier.wing_components(g, theta, 12) == 0).all()
    eu = [u for u in range(3) for _ in range(3)] + [u for u in range(3, 6) for _ in range(3)]
    ev = [v for _ in range(3) for v in range(3)] + [v for _ in range(3) for v in range(3, 6)]
    g2 = gen.from_edges(6, 6, eu, ev)
    th2 = oracle.wing(g2)
    comp = hier.wing_components(g2, th2, 1)
    assert list(comp) == [0] * 9 + [9] * 9
