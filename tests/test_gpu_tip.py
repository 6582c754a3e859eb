"""GPU parity: butterfly counts and tip numbers from the CUDA library against
the CPU oracle, bit-exact, through the C ABI (via the thin binding)."""
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


def graphs():
    out = {
        "gprime": gen.from_edges(4, 3, [0, 0, 1, 1, 1, 2, 2, 3, 3], [0, 1, 0, 1, 2, 1, 2, 1, 2]),
        "k_5_7": gen.complete(5, 7),
        "k_40_3": gen.complete(40, 3),
        "rand_30_20": rand_graph(30, 20, 0.3, 1),
        "rand_dense_60_50": rand_graph(60, 50, 0.7, 2),
        "uniform_2k_1k_20k": gen.make("uniform_2k_1k_20k"),
        "chunglu_20k_4k_200k": gen.make("chunglu_20k_4k_200k"),
        "chunglu_5k_1k_50k_planted": gen.make("chunglu_5k_1k_50k_planted"),
        "isolated": gen.from_edges(6, 5, [0, 0, 1, 1], [0, 1, 0, 1]),
    }
    return out


GRAPHS = graphs()


@pytest.mark.parametrize("name", list(GRAPHS))
def test_counts_match_oracle(pbng, name):
    g = GRAPHS[name]
    dg = pbng.to_device(g)
    cu, cv, ce = pbng.count(dg, vertices=True, edges=True)
    assert np.array_equal(pbng.as_u64(cu), oracle.vertex_counts(g, "U"))
    assert np.array_equal(pbng.as_u64(cv), oracle.vertex_counts(g, "V"))
    assert np.array_equal(pbng.as_u64(ce), oracle.edge_counts(g))


_tip_cache = {}


def oracle_tip(name, side):
    k = (name, side)
    if k not in _tip_cache:
        _tip_cache[k] = oracle.tip(GRAPHS[name], side)
    return _tip_cache[k]


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("side", ["U", "V"])
def test_tip_matches_oracle(pbng, name, side):
    g = GRAPHS[name]
    dg = pbng.to_device(g)
    got = pbng.as_u64(pbng.tip_decompose(dg, side, P=8))
    assert np.array_equal(got, oracle_tip(name, side))


@pytest.mark.parametrize("P", [1, 2, 8, 150, 10 ** 6])
@pytest.mark.parametrize("side", ["U", "V"])
def test_tip_independent_of_P(pbng, P, side):
    name = "chunglu_5k_1k_50k_planted"
    dg = pbng.to_device(GRAPHS[name])
    got = pbng.as_u64(pbng.tip_decompose(dg, side, P=P))
    assert np.array_equal(got, oracle_tip(name, side))


def test_uniform_config_tip_u_p8(pbng):
    name = "uniform_2k_1k_20k"
    dg = pbng.to_device(GRAPHS[name])
    got, st = pbng.tip_decompose(dg, "U", P=8, with_stats=True)
    assert np.array_equal(pbng.as_u64(got), oracle_tip(name, "U"))
    assert 1 <= st["parts_used"] <= 8
    assert st["rounds"] >= st["parts_used"]


@pytest.mark.parametrize("recount,compact", [(False, False), (False, True), (True, False), (True, True)])
def test_tip_optimisations_do_not_change_results(pbng, recount, compact):
    name = "chunglu_20k_4k_200k"
    dg = pbng.to_device(GRAPHS[name])
    for side in ("U", "V"):
        got = pbng.as_u64(pbng.tip_decompose(dg, side, P=40, recount=recount, compact=compact))
        assert np.array_equal(got, oracle_tip(name, side))


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("side", ["U", "V"])
def test_tip_graph_rounds_match_oracle(pbng, name, side):
    """Coarse rounds captured as a CUDA graph with a device-side WHILE loop."""
    dg = pbng.to_device(GRAPHS[name])
    for P in (1, 8, 150):
        got = pbng.as_u64(pbng.tip_decompose(dg, side, P=P, graph_rounds=True))
        assert np.array_equal(got, oracle_tip(name, side))


@pytest.mark.parametrize("compact", [False, True])
def test_tip_graph_rounds_same_work_as_host_loop(pbng, compact):
    """Without re-count both modes peel the same rounds with the same wedges."""
    name = "chunglu_20k_4k_200k"
    dg = pbng.to_device(GRAPHS[name])
    for side in ("U", "V"):
        a, sa = pbng.tip_decompose(dg, side, P=40, recount=False, compact=compact, with_stats=True)
        b, sb = pbng.tip_decompose(dg, side, P=40, recount=False, compact=compact, graph_rounds=True,
                                   with_stats=True)
        assert np.array_equal(pbng.as_u64(a), pbng.as_u64(b))
        assert np.array_equal(pbng.as_u64(b), oracle_tip(name, side))
        for k in ("rounds", "wedges_cd", "parts_used", "updates"):
            assert sa[k] == sb[k], k


_BK_GRAPH = {}


def bucket_graph():
    """80k x 4k Chung-Lu graph: the peeled side spans several target buckets."""
    if not _BK_GRAPH:
        g = gen.chung_lu(80000, 4000, 300000, 2.3, 2.3, 2000, seed=77)
        _BK_GRAPH["g"], _BK_GRAPH["U"] = g, oracle.tip(g, "U")
    return _BK_GRAPH["g"], _BK_GRAPH["U"]


@pytest.mark.parametrize("shift", [0, 15, 16, 17])
@pytest.mark.parametrize("graph_rounds", [False, True])
def test_tip_bucket_widths(pbng, shift, graph_rounds):
    """Target buckets of 2^14 ids (dense passes), and wider buckets whose heavy
    passes are cut into dense sub-ranges, with and without compaction."""
    g, want = bucket_graph()
    dg = pbng.to_device(g)
    for compact in (True, False):
        got = pbng.as_u64(pbng.tip_decompose(dg, "U", P=30, bucket_shift=shift, compact=compact,
                                             graph_rounds=graph_rounds))
        assert np.array_equal(got, want)


def repeat_graph():
    """200k x 1k graph whose vertices share two neighbours in blocks of 5000:
    one block inside a single 2^14-id bucket, one spread over all buckets."""
    if "rep" not in _BK_GRAPH:
        rng = np.random.default_rng(91)
        nu, nv = 200000, 1000
        eu = [np.arange(nu), np.arange(0, nu, 3)]
        ev = [rng.integers(4, nv, size=nu), rng.integers(4, nv, size=len(range(0, nu, 3)))]
        for S, ys in ((np.arange(100, 5100), (0, 1)), (np.arange(0, nu, 40)[:5000], (2, 3))):
            for y in ys:
                eu.append(S)
                ev.append(np.full(S.size, y))
        key = np.unique(np.concatenate(eu).astype(np.int64) * nv + np.concatenate(ev))
        g = gen.from_edges(nu, nv, key // nv, key % nv)
        _BK_GRAPH["rep"] = (g, oracle.tip(g, "U"))
    return _BK_GRAPH["rep"]


@pytest.mark.parametrize("shift", [0, 17])
@pytest.mark.parametrize("graph_rounds", [False, True])
def test_tip_many_repeated_targets(pbng, shift, graph_rounds):
    """Block-class vertices whose targets are mostly shared (c >= 2) within
    one bucket, and spread over all buckets."""
    g, want = repeat_graph()
    dg = pbng.to_device(g)
    for P in (1, 12):
        got = pbng.as_u64(pbng.tip_decompose(dg, "U", P=P, bucket_shift=shift, graph_rounds=graph_rounds))
        assert np.array_equal(got, want)


def hub_graph():
    """One U vertex adjacent to all 70k V vertices (2^16 or more neighbours:
    32-bit dense counters, neighbours read in chunks), 20k U vertices."""
    if "hub" not in _BK_GRAPH:
        rng = np.random.default_rng(5)
        nu, nv = 20000, 70000
        eu = [np.zeros(nv, np.int64)] + [rng.integers(1, nu, size=nv) for _ in range(2)]
        ev = [np.arange(nv)] * 3
        key = np.unique(np.concatenate(eu) * nv + np.concatenate(ev))
        g = gen.from_edges(nu, nv, key // nv, key % nv)
        _BK_GRAPH["hub"] = (g, oracle.tip(g, "U"))
    return _BK_GRAPH["hub"]


@pytest.mark.parametrize("graph_rounds", [False, True])
def test_tip_hub_vertex(pbng, graph_rounds):
    g, want = hub_graph()
    dg = pbng.to_device(g)
    for P in (1, 3, 30):
        got = pbng.as_u64(pbng.tip_decompose(dg, "U", P=P, graph_rounds=graph_rounds))
        assert np.array_equal(got, want)


def test_tip_explicit_and_random_bounds(pbng):
    name = "chunglu_20k_4k_200k"
    g = GRAPHS[name]
    dg = pbng.to_device(g)
    want = oracle_tip(name, "U")
    rng = np.random.default_rng(7)
    for trial in range(4):
        hi = int(want.max()) + 2
        b = np.unique(rng.integers(1, hi, size=int(rng.integers(1, 30)))).astype(np.uint64)
        got = pbng.as_u64(pbng.tip_decompose(dg, "U", P=len(b) + 1, bounds=b))
        assert np.array_equal(got, want)
    # bounds at the exact tip-number levels, and bounds far below the minimum
    lv = np.unique(want)[1:].astype(np.uint64)
    got = pbng.as_u64(pbng.tip_decompose(dg, "U", P=len(lv) + 1, bounds=lv))
    assert np.array_equal(got, want)


def test_tip_host_buffers(pbng):
    name = "chunglu_5k_1k_50k_planted"
    got = pbng.tip_decompose_host(GRAPHS[name], "V", P=20)
    assert np.array_equal(got, oracle_tip(name, "V"))


def test_batch_matches_individual(pbng):
    gs = [gen.batch_graph(1000 + i, scale=0.05) for i in range(12)] + [GRAPHS["gprime"], GRAPHS["isolated"]]
    dgs = [pbng.to_device(g) for g in gs]
    res = pbng.tip_decompose_batch(dgs, "U", P=30)
    for g, r in zip(gs, res):
        assert np.array_equal(pbng.as_u64(r), oracle.tip(g, "U"))
    res = pbng.tip_decompose_batch(dgs, "V", P=5)
    for g, r in zip(gs, res):
        assert np.array_equal(pbng.as_u64(r), oracle.tip(g, "V"))


def test_empty_graphs(pbng):
    import torch
    g = gen.from_edges(3, 4, [], [])
    dg = pbng.to_device(g)
    assert (pbng.as_u64(pbng.tip_decompose(dg, "U", P=4)) == 0).all()
    cu, cv, ce = pbng.count(dg, vertices=True, edges=True)
    assert (pbng.as_u64(cu) == 0).all() and (pbng.as_u64(cv) == 0).all() and ce.numel() == 0


def test_malformed_csr_is_rejected(pbng):
    import torch
    cases = {
        "unsorted": ([0, 3, 4], [2, 0, 1, 1]),
        "duplicate": ([0, 2, 3], [1, 1, 0]),
        "out_of_range": ([0, 1, 2], [0, 9]),
        "bad_offsets": ([0, 3, 2], [0, 1, 2]),
    }
    for name, (off, adj) in cases.items():
        dg = pbng.DeviceGraph(2, 3, torch.tensor(off, dtype=torch.int64, device="cuda"),
                              torch.tensor(adj, dtype=torch.int32, device="cuda"))
        with pytest.raises(pbng.PbngError) as ei:
            pbng.tip_decompose(dg, "U", P=2)
        assert ei.value.code == pbng.PBNG_EINVAL, name


@pytest.mark.parametrize("knob,value", [("warp_max_w", 1), ("warp_max_w", 128), ("group_max_w", 512),
                                        ("item_w", 4096), ("item_w", 1 << 30), ("bucket_shift", 14), ("bucket_shift", 16),
                                        ("graph_rounds", True), ("count_scratch", 1), ("count_scratch", 2),
                                        ("fd_cluster_min", 8192), ("fd_cluster_min", 0xFFFFFFFF)])
def test_tip_every_schedule_variant(pbng, knob, value):
    """Every value the autotuner may choose, forced once: identical tip numbers."""
    from paper_2110_12511_gb300 import autotune as at
    cfg = dict(at.DEFAULT)
    cfg[knob] = value
    if knob == "group_max_w":
        cfg["warp_max_w"] = 256
    for name in ("chunglu_5k_1k_50k_planted", "chunglu_20k_4k_200k"):
        dg = pbng.to_device(GRAPHS[name])
        for side in ("U", "V"):
            got = pbng.as_u64(pbng.tip_decompose(dg, side, P=20, **at.split(cfg)))
            assert np.array_equal(got, oracle_tip(name, side))
    g, want = bucket_graph()
    got = pbng.as_u64(pbng.tip_decompose(pbng.to_device(g), "U", P=20, **at.split(cfg)))
    assert np.array_equal(got, want)


def test_autotuner_choice_gives_identical_numbers(pbng, tmp_path):
    from paper_2110_12511_gb300 import autotune as at
    name = "chunglu_20k_4k_200k"
    dg = pbng.to_device(GRAPHS[name])
    cache = str(tmp_path / "tune.json")
    cfg, t, table = at.tune_tip(dg, "U", P=40, reps=1, cache=cache)
    assert at.valid(cfg) and t > 0 and len(table) >= 2
    got = pbng.as_u64(pbng.tip_decompose(dg, "U", P=40, **at.split(cfg)))
    assert np.array_equal(got, oracle_tip(name, "U"))
    cfg2, t2, table2 = at.tune_tip(dg, "U", P=40, cache=cache)  # from the cache
    assert cfg2 == cfg and table2 == []
    gs = [gen.batch_graph(1000 + i, scale=0.05) for i in range(8)]
    size, tb = at.tune_batch([pbng.to_device(g) for g in gs], "U", P=20, sizes=(2, 8), cfg=cfg)
    assert size in (2, 8) and len(tb) == 2


def recount_bound(g, side):
    """Smallest first bound whose active set (every vertex with initial count
    below it) has more wedges than the counting bound sum_e min(d_u, d_v):
    the round re-counts the remaining vertices instead of peeling (Sec. 5.1)."""
    h = g if side == "U" else g.swapped()
    du = np.diff(h.u_off).astype(np.int64)
    dv = np.bincount(h.u_adj, minlength=h.nv).astype(np.int64)
    eu = np.repeat(np.arange(h.nu), du)
    wbound = int(np.minimum(du[eu], dv[h.u_adj]).sum())
    W = np.bincount(eu, weights=dv[h.u_adj], minlength=h.nu)
    cnt = oracle.vertex_counts(g, side)
    order = np.argsort(cnt, kind="stable")
    k = int(np.searchsorted(np.cumsum(W[order]), wbound, side="right"))
    assert k < h.nu, "no first round exceeds the counting bound on this graph"
    return int(cnt[order[k]]) + 1, wbound


@pytest.mark.parametrize("side", ["U", "V"])
def test_tip_recount_branch_runs(pbng, side):
    """Sec. 5.1: the first round's active vertices have more wedges than the
    counting bound, so the round re-counts the remaining vertices; the tip
    numbers still equal the oracle's, and without re-count nothing is re-counted."""
    name = "chunglu_20k_4k_200k"
    g = GRAPHS[name]
    dg = pbng.to_device(g)
    b0, wbound = recount_bound(g, side)
    bounds = np.array([b0, 2 * b0, 4 * b0], dtype=np.uint64)
    got, st = pbng.tip_decompose(dg, side, P=5, bounds=bounds, recount=True, with_stats=True)
    assert st["wedge_bound"] == wbound
    assert st["recounts"] > 0
    assert np.array_equal(pbng.as_u64(got), oracle_tip(name, side))
    got2, st2 = pbng.tip_decompose(dg, side, P=5, bounds=bounds, recount=False, with_stats=True)
    assert st2["recounts"] == 0
    assert np.array_equal(pbng.as_u64(got2), oracle_tip(name, side))
    assert st["wedges_cd"] < st2["wedges_cd"]  # the re-count replaced a heavier peel


@pytest.mark.parametrize("side", ["U", "V"])
@pytest.mark.parametrize("P", [1, 8, 40])
def test_propose_bounds_reproduce_the_ranges(pbng, side, P):
    """pbng_propose_bounds returns theta(1..P+1) of the coarse phase
    (Sec. 3.1.3); fed back as explicit bounds they give the same ranges and
    the oracle's tip numbers (Sec. 4.1 Th. 2)."""
    name = "chunglu_20k_4k_200k"
    dg = pbng.to_device(GRAPHS[name])
    b = pbng.propose_bounds(dg, side, P=P)
    assert b.size == P + 1 and b[0] == 0 and b[-1] == np.iinfo(np.uint64).max
    inner = b[1:][b[1:] != np.iinfo(np.uint64).max]
    assert np.all(np.diff(inner.astype(np.float64)) > 0)
    used = np.zeros(P + 1, dtype=np.uint64)
    th, st = pbng.tip_decompose(dg, side, P=P, with_stats=True, bounds_out=used)
    assert inner.size in (st["parts_used"] - 1, st["parts_used"])
    assert np.array_equal(used[:inner.size], inner) and not used[inner.size:].any()
    th2, st2 = pbng.tip_decompose(dg, side, P=P, bounds=inner, with_stats=True)
    assert np.array_equal(pbng.as_u64(th2), oracle_tip(name, side))
    assert st2["parts_used"] == st["parts_used"]


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("cmin", [1, 0xFFFFFFFF])
def test_tip_cluster_fine_phase(pbng, name, cmin):
    """Fine phase with every partition peeled by a thread-block cluster
    (cmin = 1: selection across blocks, warps of all blocks on light
    vertices, heavy vertices counted in counters spread over the blocks'
    shared memory) or by single blocks only: the oracle's numbers."""
    dg = pbng.to_device(GRAPHS[name])
    for side in ("U", "V"):
        for P in (1, 8):
            got = pbng.tip_decompose(dg, side, P=P, schedule={"fd_cluster_min": cmin})
            assert np.array_equal(pbng.as_u64(got), oracle_tip(name, side))


def test_tip_cluster_fine_phase_global_counters(pbng):
    """A 270k-vertex partition (more than a cluster's shared counters hold):
    the heavy vertices count in global memory; numbers equal the oracle's."""
    g = gen.uniform(270000, 2000, 700000, 41)
    dg = pbng.to_device(g)
    got, st = pbng.tip_decompose(dg, "U", P=1, schedule={"fd_cluster_min": 1}, with_stats=True)
    assert st["parts_used"] == 1
    assert np.array_equal(pbng.as_u64(got), oracle.tip(g, "U"))


def tier_graph():
    """Disjoint bicliques: the U vertices of each size tie, so one fine-phase
    step peels all of them, with in-partition wedge counts of 380 (128-thread
    groups take them), 1,560 and 3,540 (single blocks of a cluster) and 5,960
    (the whole cluster); the last step (K_80,80) makes no updates.  Plus a
    sparse random part on vertices of its own."""
    rng = np.random.default_rng(77)
    eu, ev, u0, v0 = [], [], 0, 0
    for a, b in ((20, 20), (20, 20), (40, 40), (40, 40), (40, 40), (60, 60), (60, 60), (150, 40), (80, 80)):
        eu.append(np.repeat(np.arange(u0, u0 + a), b))
        ev.append(np.tile(np.arange(v0, v0 + b), a))
        u0, v0 = u0 + a, v0 + b
    eu.append(u0 + rng.integers(0, 300, 1500))
    ev.append(v0 + rng.integers(0, 100, 1500))
    return gen.from_edges(u0 + 300, v0 + 100, np.concatenate(eu), np.concatenate(ev))


@pytest.mark.parametrize("cmin", [1, 0xFFFFFFFF])
def test_tip_fine_phase_heavy_tiers(pbng, tmp_path, cmin):
    """A step that peels many heavy vertices at once: 128-thread groups take
    the lighter ones, then (on a thread-block cluster) single blocks, and the
    whole team the rest (per the fine-phase trace); one block per partition
    has no block tier.  Numbers equal the oracle's either way."""
    import os
    g = tier_graph()
    dg = pbng.to_device(g)
    tr = tmp_path / "trace.txt"
    os.environ["PBNG_TRACE"] = str(tr)
    try:
        got = pbng.tip_decompose(dg, "U", P=1, schedule={"fd_cluster_min": cmin})
    finally:
        del os.environ["PBNG_TRACE"]
    assert np.array_equal(pbng.as_u64(got), oracle.tip(g, "U"))
    rows = [list(map(int, l.split()[1:])) for l in open(tr) if l.startswith("F ")]
    assert len(rows) == 1
    heavy, by_block, by_team = rows[0][-3:]
    if cmin == 1:
        assert by_block > 0 and by_team > 0 and heavy > by_block + by_team
    else:
        assert by_block == 0 and 0 < by_team < heavy


@pytest.mark.parametrize("scratch", [0, 1, 2, 3])
@pytest.mark.parametrize("name", ["chunglu_20k_4k_200k", "chunglu_5k_1k_50k_planted", "rand_dense_60_50", "bucket"])
def test_counts_every_scratch_kind(pbng, name, scratch):
    """Alg. 1 with every scratch-counter kind of the heavier starts (automatic,
    shared hashes first, dense only, dense with 32-bit label chunks): counts
    equal the oracle's; the 80k x 4k graph has more than 2^15 labels, so its
    dense chunks start at label 0 and 32768 (16384 steps with 32-bit)."""
    g = bucket_graph()[0] if name == "bucket" else GRAPHS[name]
    dg = pbng.to_device(g)
    cu, cv, ce = pbng.count(dg, vertices=True, edges=True, scratch=scratch)
    assert np.array_equal(pbng.as_u64(cu), oracle.vertex_counts(g, "U"))
    assert np.array_equal(pbng.as_u64(cv), oracle.vertex_counts(g, "V"))
    assert np.array_equal(pbng.as_u64(ce), oracle.edge_counts(g))


@pytest.mark.parametrize("scratch", [1, 2, 3])
def test_tip_every_scratch_kind(pbng, scratch):
    """The initial counts and the re-counts of a decomposition with each
    scratch kind (re-count forced as in test_tip_recount_branch_runs)."""
    name = "chunglu_20k_4k_200k"
    dg = pbng.to_device(GRAPHS[name])
    for side in ("U", "V"):
        b0, _ = recount_bound(GRAPHS[name], side)
        got, st = pbng.tip_decompose(dg, side, P=5, bounds=np.array([b0, 2 * b0], dtype=np.uint64),
                                     schedule={"count_scratch": scratch}, with_stats=True)
        assert st["recounts"] > 0
        assert np.array_equal(pbng.as_u64(got), oracle_tip(name, side))
