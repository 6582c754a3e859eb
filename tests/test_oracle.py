"""Pins for the CPU oracle (no GPU).

The oracle is checked against facts that do not come from itself:
4-tuple butterfly enumeration, the common-neighbour matrix A A^T, the closed
forms of complete bipartite graphs, the worked example G' described in
Sec. 2.3 / Sec. 3.3.3, subset and fixed-point restatements of Def. 1-2, and
invariants (sum of U counts = 2 x total, of V counts = 2 x total, of edge
counts = 4 x total; theta <= initial count).
"""
import json
import os
from math import comb

import numpy as np
import pytest

import bigraph_gen as gen
import oracle
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_graph(nu, nv, p, seed):
    rng = np.random.default_rng(seed)
    a = rng.random((nu, nv)) < p
    eu, ev = np.nonzero(a)
    return gen.from_edges(nu, nv, eu, ev)


TINY = [(nu, nv, p, s) for s, (nu, nv, p) in enumerate(
    [(4, 4, 0.6), (5, 4, 0.7), (6, 5, 0.5), (7, 6, 0.6), (8, 5, 0.8), (9, 7, 0.45), (6, 9, 0.5),
     (8, 8, 0.35), (3, 10, 0.9), (10, 3, 0.9)])]


@pytest.mark.parametrize("nu,nv,p,seed", TINY)
def test_counts_match_enumeration(nu, nv, p, seed):
    g = rand_graph(nu, nv, p, seed)
    cu, cv, ce, total = brute.counts_by_enumeration(g)
    assert np.array_equal(oracle.vertex_counts(g, "U").astype(np.int64), cu)
    assert np.array_equal(oracle.vertex_counts(g, "V").astype(np.int64), cv)
    assert np.array_equal(oracle.edge_counts(g).astype(np.int64), ce)
    assert cu.sum() == 2 * total and cv.sum() == 2 * total and ce.sum() == 4 * total


@pytest.mark.parametrize("seed", range(4))
def test_counts_match_common_neighbour_matrix(seed):
    g = rand_graph(60, 40, 0.25, 100 + seed)
    b = brute.pair_butterflies(g)
    cu = b.sum(axis=1)
    assert np.array_equal(oracle.vertex_counts(g, "U").astype(np.int64), cu)
    total = b.sum() // 2
    cv = oracle.vertex_counts(g, "V").astype(np.int64)
    ce = oracle.edge_counts(g).astype(np.int64)
    assert cv.sum() == 2 * total and ce.sum() == 4 * total
    # per edge: sum over u' in N_v \ {u} of (c(u,u') - 1)
    a = brute.adjacency(g)
    c = a @ a.T
    eu, ev = g.edges()
    for e in range(0, g.m, 7):
        u, v = int(eu[e]), int(ev[e])
        others = [w for w in np.nonzero(a[:, v])[0] if w != u]
        assert ce[e] == sum(int(c[u, w]) - 1 for w in others)


@pytest.mark.parametrize("a,b", [(2, 2), (2, 5), (3, 3), (4, 7), (7, 4), (1, 6), (9, 9)])
def test_complete_bipartite_closed_forms(a, b):
    g = gen.complete(a, b)
    cu = (a - 1) * comb(b, 2)
    cv = (b - 1) * comb(a, 2)
    ce = (a - 1) * (b - 1)
    assert (oracle.vertex_counts(g, "U") == cu).all()
    assert (oracle.vertex_counts(g, "V") == cv).all()
    assert (oracle.edge_counts(g) == ce).all()
    assert (oracle.tip(g, "U") == cu).all()
    assert (oracle.tip(g, "V") == cv).all()
    assert (oracle.wing(g) == ce).all()


def load_gprime():
    with open(os.path.join(GOLDEN, "gprime.json")) as f:
        d = json.load(f)
    names = [e[0] for e in d["edges"]]
    g = gen.from_edges(d["nu"], d["nv"], [e[1] for e in d["edges"]], [e[2] for e in d["edges"]])
    # from_edges sorts by (u, v); the listed order is already sorted
    eu, ev = g.edges()
    assert [(int(u), int(v)) for u, v in zip(eu, ev)] == [(e[1], e[2]) for e in d["edges"]]
    return g, names, d


def test_gprime_worked_example():
    g, names, d = load_gprime()
    h = d["derived_by_hand"]
    ce = oracle.edge_counts(g)
    assert int(ce[names.index("e3")]) == d["printed"]["edge_count_e3"]
    assert [int(x) for x in ce] == [h["edge_counts"][n] for n in names]
    assert [int(x) for x in oracle.vertex_counts(g, "U")] == h["u_counts"]
    assert [int(x) for x in oracle.vertex_counts(g, "V")] == h["v_counts"]
    assert [int(x) for x in oracle.wing(g)] == [h["wing_numbers"][n] for n in names]
    assert [int(x) for x in oracle.tip(g, "U")] == h["tip_u"]
    assert [int(x) for x in oracle.tip(g, "V")] == h["tip_v"]
    # bloom B1 (dominant {v1, v2}, non-dominant {u1, u2, u3}) holds C(3,2) butterflies
    assert comb(d["printed"]["bloom_numbers"]["B1"], 2) == d["printed"]["butterflies_in_B1"]


@pytest.mark.parametrize("nu,nv,p,seed", TINY[:8])
def test_tip_matches_subset_definition(nu, nv, p, seed):
    g = rand_graph(nu, nv, p, seed)
    assert np.array_equal(oracle.tip(g, "U").astype(np.int64), brute.tip_by_subsets(g))
    if nv <= 9:
        assert np.array_equal(oracle.tip(g, "V").astype(np.int64), brute.tip_by_subsets(g.swapped()))


@pytest.mark.parametrize("seed", range(6))
def test_wing_matches_subset_definition(seed):
    rng = np.random.default_rng(500 + seed)
    for _ in range(50):
        g = rand_graph(int(rng.integers(3, 6)), int(rng.integers(3, 6)), 0.7, int(rng.integers(1 << 30)))
        if 4 <= g.m <= 13:
            break
    assert np.array_equal(oracle.wing(g).astype(np.int64), brute.wing_by_subsets(g))


@pytest.mark.parametrize("seed", range(5))
def test_tip_matches_fixpoint(seed):
    g = rand_graph(80, 30, 0.2 + 0.05 * seed, 200 + seed)
    assert np.array_equal(oracle.tip(g, "U").astype(np.int64), brute.tip_by_fixpoint(g))
    assert np.array_equal(oracle.tip(g, "V").astype(np.int64), brute.tip_by_fixpoint(g.swapped()))


@pytest.mark.parametrize("seed", range(4))
def test_wing_matches_fixpoint(seed):
    g = rand_graph(14, 12, 0.3 + 0.05 * seed, 300 + seed)
    assert np.array_equal(oracle.wing(g).astype(np.int64), brute.wing_by_fixpoint(g))


def test_planted_powerlaw_small_fixpoint():
    g = gen.chung_lu(40, 25, 220, 2.2, 2.4, 20, seed=77, nplant=2, plant_lo=4, plant_hi=7)
    assert np.array_equal(oracle.tip(g, "U").astype(np.int64), brute.tip_by_fixpoint(g))
    assert np.array_equal(oracle.wing(g).astype(np.int64), brute.wing_by_fixpoint(g))


def test_theta_bounded_by_count_and_edge_cases():
    g = gen.make("chunglu_5k_1k_50k_planted")
    cnt = oracle.vertex_counts(g, "U")
    th = oracle.tip(g, "U")
    assert (th <= cnt).all()
    # isolated vertices and empty graphs
    e = gen.from_edges(5, 3, [], [])
    assert (oracle.tip(e, "U") == 0).all() and oracle.wing(e).shape == (0,)
    star = gen.from_edges(1, 6, [0] * 6, range(6))
    assert (oracle.tip(star, "U") == 0).all() and (oracle.wing(star) == 0).all()


def test_support_within_matches_definition():
    g = rand_graph(30, 20, 0.3, 9)
    t = oracle.Transposed(g)
    b = brute.pair_butterflies(g)
    rng = np.random.default_rng(3)
    member = rng.random(g.nu) < 0.6
    for u in range(g.nu):
        assert t.vertex_support_within(member, u) == int(b[u, member & (np.arange(g.nu) != u)].sum())
    bfs = brute._edge_butterflies(g)
    emember = rng.random(g.m) < 0.7
    for e in range(g.m):
        want = sum(1 for bf in bfs if e in bf and all(emember[x] for x in bf if x != e))
        assert t.edge_support_within(emember, e) == want


def test_parallel_vertex_counts_equal_sequential():
    """The all-cores counting used for the CPU baseline computes the same
    definition as vertex_counts (Sec. 2.1), on both sides."""
    for g in (gen.make("chunglu_5k_1k_50k_planted"), gen.complete(7, 5), gen.from_edges(3, 2, [], [])):
        for side in ("U", "V"):
            got, threads = oracle.vertex_counts_parallel(g, side)
            assert threads >= 1
            assert np.array_equal(got, oracle.vertex_counts(g, side))
