"""GPU parity: wing numbers (BE-Index PBNG) against the CPU oracle's
bottom-up peeling, bit-exact, for several graphs, partition counts, bounds
and with the dynamic list compaction on and off."""
import numpy as np
import pytest

import bigraph_gen as gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pbng():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_12511_gb300 import build as b
    b.build()
    import paper_2110_12511_gb300 as m
    m.lib()
    return m


def rand_graph(nu, nv, p, seed):
    rng = np.random.default_rng(seed)
    a = rng.random((nu, nv)) < p
    eu, ev = np.nonzero(a)
    return gen.from_edges(nu, nv, eu, ev)


GRAPHS = {
    "gprime": gen.from_edges(4, 3, [0, 0, 1, 1, 1, 2, 2, 3, 3], [0, 1, 0, 1, 2, 1, 2, 1, 2]),
    "k_6_5": gen.complete(6, 5),
    "k_2_30": gen.complete(2, 30),
    "rand_40_30": rand_graph(40, 30, 0.3, 11),
    "rand_dense_50_40": rand_graph(50, 40, 0.6, 12),
    "uniform_2k_1k_20k": gen.make("uniform_2k_1k_20k"),
    "planted_small": gen.chung_lu(3000, 600, 12000, 2.2, 2.4, 500, seed=31, nplant=8, plant_lo=6, plant_hi=25),
    "chunglu_5k_1k_50k_planted": gen.make("chunglu_5k_1k_50k_planted"),
    "isolated": gen.from_edges(6, 5, [0, 0, 1, 1], [0, 1, 0, 1]),
}
_cache = {}


def oracle_wing(name):
    if name not in _cache:
        _cache[name] = oracle.wing(GRAPHS[name])
    return _cache[name]


@pytest.mark.parametrize("name", list(GRAPHS))
def test_wing_matches_oracle(pbng, name):
    dg = pbng.to_device(GRAPHS[name])
    got, st = pbng.wing_decompose(dg, P=16, with_stats=True)
    assert np.array_equal(pbng.as_u64(got), oracle_wing(name))


@pytest.mark.parametrize("name", list(GRAPHS))
def test_be_index_properties(pbng, name):
    """Sec. 2.3 Property 1-2 on the BE-Index the wing path builds: every
    butterfly lies in exactly one maximal priority bloom, which holds C(k_B, 2)
    of them, and an edge of bloom B lies in k_B - 1 of B's butterflies; so the
    per-edge sums over blooms equal the oracle's edge counts and the sum over
    blooms equals the oracle's total (sum of edge counts / 4 = sum of U-vertex
    counts / 2)."""
    g = GRAPHS[name]
    dg = pbng.to_device(g)
    (per_edge, total), st = pbng.be_index_sums(dg, with_stats=True)
    ce = oracle.edge_counts(g)
    assert np.array_equal(pbng.as_u64(per_edge), ce)
    butterflies = int(ce.sum(dtype=np.uint64)) // 4
    assert total == butterflies
    assert 2 * total == int(oracle.vertex_counts(g, "U").sum(dtype=np.uint64))
    # and the decomposition runs on an index of the same size
    _, sw = pbng.wing_decompose(dg, P=16, with_stats=True)
    assert (st["links"], st["blooms"]) == (sw["links"], sw["blooms"])


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("cmin", [1, 0xFFFFFFFF])
def test_wing_cluster_fine_phase(pbng, name, cmin):
    """Fine phase with every partition peeled by a thread-block cluster
    (cmin = 1) or by single blocks only: the oracle's numbers either way."""
    dg = pbng.to_device(GRAPHS[name])
    for P in (1, 16):
        got = pbng.wing_decompose(dg, P=P, schedule={"fd_cluster_min": cmin})
        assert np.array_equal(pbng.as_u64(got), oracle_wing(name))


@pytest.mark.parametrize("P", [1, 2, 7, 100, 10 ** 6])
def test_wing_independent_of_P(pbng, P):
    name = "planted_small"
    dg = pbng.to_device(GRAPHS[name])
    assert np.array_equal(pbng.as_u64(pbng.wing_decompose(dg, P=P)), oracle_wing(name))


@pytest.mark.parametrize("compact", [False, True])
def test_wing_compaction_does_not_change_results(pbng, compact):
    name = "chunglu_5k_1k_50k_planted"
    dg = pbng.to_device(GRAPHS[name])
    assert np.array_equal(pbng.as_u64(pbng.wing_decompose(dg, P=50, compact=compact)), oracle_wing(name))


def test_wing_random_bounds(pbng):
    name = "planted_small"
    want = oracle_wing(name)
    dg = pbng.to_device(GRAPHS[name])
    rng = np.random.default_rng(5)
    for _ in range(4):
        b = np.unique(rng.integers(1, int(want.max()) + 3, size=int(rng.integers(1, 25)))).astype(np.uint64)
        assert np.array_equal(pbng.as_u64(pbng.wing_decompose(dg, P=len(b) + 1, bounds=b)), want)


def test_wing_counts_match_edge_counts(pbng):
    # the per-edge counts behind the initial supports equal pbng_count's
    name = "planted_small"
    g = GRAPHS[name]
    dg = pbng.to_device(g)
    ce = pbng.as_u64(pbng.count(dg, vertices=False, edges=True)[2])
    assert np.array_equal(ce, oracle.edge_counts(g))
    w = pbng.as_u64(pbng.wing_decompose(dg, P=10))
    assert (w <= ce).all()


def test_wing_batch_matches_oracle(pbng):
    """Many graphs in one call: every graph's wing numbers equal the oracle's."""
    names = list(GRAPHS)
    gs = [GRAPHS[n] for n in names] + [gen.batch_graph(2000 + i, scale=0.02) for i in range(6)]
    empty = gen.from_edges(3, 2, [], [])
    gs.append(empty)
    dgs = [pbng.to_device(g) for g in gs]
    got = pbng.wing_decompose_batch(dgs, P=30)
    for g, n, w in zip(gs, names + [None] * 7, got):
        want = oracle_wing(n) if n is not None else oracle.wing(g)
        assert np.array_equal(pbng.as_u64(w), want)


@pytest.mark.parametrize("scratch", [1, 2, 3])
def test_wing_every_scratch_kind(pbng, scratch):
    """The per-edge counts and BE-Index sizes behind the wing numbers with
    each scratch-counter kind."""
    name = "chunglu_5k_1k_50k_planted"
    dg = pbng.to_device(GRAPHS[name])
    got = pbng.wing_decompose(dg, P=20, schedule={"count_scratch": scratch})
    assert np.array_equal(pbng.as_u64(got), oracle_wing(name))
