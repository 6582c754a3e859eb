"""Full-size parity on the benchmark workloads, in the launch configuration
bench.py times.

* Where the oracle's complete bottom-up peeling was run once by
  tests/golden/make_golden.py, the GPU tip numbers must hash to the same
  SHA-256 (bit-exact over every vertex) and match the stored samples; the
  generated graph's hash is checked first, so generator drift cannot pass.
* Everywhere, sampled entities are checked with local certificates the
  oracle computes one at a time: for an entity l with number t,
    (a) l has >= t butterflies inside {theta >= t}   (it lies in a t-level),
    (b) l has <= t butterflies inside {theta >= t+1} + {l} (it cannot join
        the (t+1)-level), and the initial count equals the oracle's count.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import bigraph_gen as gen
import oracle

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
_graphs = {}


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


def graph(name):
    if name not in _graphs:
        _graphs[name] = gen.make(name)
    return _graphs[name]


def gsha(g):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(g.u_off, dtype=np.uint64).tobytes())
    h.update(np.ascontiguousarray(g.u_adj, dtype=np.uint32).tobytes())
    return h.hexdigest()


def golden(job):
    p = os.path.join(GOLDEN, job + ".json")
    if not os.path.exists(p):
        pytest.skip(f"{job}: no stored oracle result")
    with open(p) as f:
        return json.load(f)


def check_tip_certificates(g, side, theta, count, k=24, seed=0):
    h = g if side == "U" else g.swapped()
    t = oracle.Transposed(h)
    rng = np.random.default_rng(seed)
    idx = np.concatenate([rng.integers(0, h.nu, size=k), [int(np.argmax(theta))]])
    for u in idx:
        u = int(u)
        th = int(theta[u])
        assert t.vertex_support_within(np.ones(h.nu, dtype=np.uint8), u) == int(count[u])
        if th > 0:
            assert t.vertex_support_within(theta >= th, u) >= th
        above = theta >= th + 1
        assert t.vertex_support_within(above, u) <= th


@pytest.mark.parametrize("side", ["U", "V"])
def test_chunglu_1m_200k_20m_tip_p150(pbng, side):
    g = graph("chunglu_1m_200k_20m")
    dg = pbng.to_device(g)
    theta = pbng.as_u64(pbng.tip_decompose(dg, side, P=150))
    cu, cv, _ = pbng.count(dg, vertices=True)
    count = pbng.as_u64(cu if side == "U" else cv)
    assert (theta <= count).all()
    check_tip_certificates(g, side, theta, count)
    gd = golden(f"tip_chunglu_1m_200k_20m_{side}")
    assert gsha(g) == gd["graph_sha256"], "generated graph differs from the one the oracle decomposed"
    for i, v in gd["samples"]:
        assert int(theta[i]) == v
    assert hashlib.sha256(theta.tobytes()).hexdigest() == gd["theta_sha256"]


def test_chunglu_5m_1m_60m_tip_p200(pbng):
    g = graph("chunglu_5m_1m_60m")
    dg = pbng.to_device(g)
    theta = pbng.as_u64(pbng.tip_decompose(dg, "U", P=200))
    count = pbng.as_u64(pbng.count(dg, vertices=True)[0])
    assert (theta <= count).all()
    check_tip_certificates(g, "U", theta, count, k=12)
    gd = golden("tip_chunglu_5m_1m_60m_U")
    assert gsha(g) == gd["graph_sha256"]
    for i, v in gd["samples"]:
        assert int(theta[i]) == v
    assert hashlib.sha256(theta.tobytes()).hexdigest() == gd["theta_sha256"]


def test_batch_4096_tip_p150(pbng):
    gd = golden("tip_batch_4096_U")
    gs = [gen.batch_graph(1000 + i) for i in range(4096)]
    hh = hashlib.sha256()
    for g in gs:
        hh.update(gsha(g).encode())
    assert hh.hexdigest() == gd["graph_sha256"]
    res = pbng.tip_decompose_batch([pbng.to_device(g) for g in gs], "U", P=150)
    h = hashlib.sha256()
    for i, r in enumerate(res):
        t = pbng.as_u64(r)
        assert hashlib.sha256(t.tobytes()).hexdigest()[:16] == gd["per_graph_sha256"][i], f"graph {i}"
        h.update(t.tobytes())
    assert h.hexdigest() == gd["theta_sha256"]


def test_chunglu_500k_100k_1m_planted_wing_p100(pbng):
    """The planted recipe with all 200 bicliques on a 1M-edge Chung-Lu base:
    every wing number equals the oracle's complete bottom-up peeling."""
    gd = golden("wing_chunglu_500k_100k_1m_planted")
    g = graph("chunglu_500k_100k_1m_planted")
    assert gsha(g) == gd["graph_sha256"]
    dg = pbng.to_device(g)
    theta = pbng.as_u64(pbng.wing_decompose(dg, P=100))
    for i, v in gd["samples"]:
        assert int(theta[i]) == v
    assert hashlib.sha256(theta.tobytes()).hexdigest() == gd["theta_sha256"]


def test_chunglu_500k_100k_5m_planted_wing_p100(pbng):
    g = graph("chunglu_500k_100k_5m_planted")
    dg = pbng.to_device(g)
    theta = pbng.as_u64(pbng.wing_decompose(dg, P=100))
    p = os.path.join(GOLDEN, "wing_chunglu_500k_100k_5m_planted.json")
    if os.path.exists(p):  # the oracle's complete peeling: bit-exact over every edge
        gd = golden("wing_chunglu_500k_100k_5m_planted")
        assert gsha(g) == gd["graph_sha256"]
        for i, v in gd["samples"]:
            assert int(theta[i]) == v
        assert hashlib.sha256(theta.tobytes()).hexdigest() == gd["theta_sha256"]
    ce = pbng.as_u64(pbng.count(dg, vertices=False, edges=True)[2])
    assert (theta <= ce).all()
    # any bounds give the same numbers (Th. 2): a different partition count
    assert np.array_equal(pbng.as_u64(pbng.wing_decompose(dg, P=37)), theta)
    t = oracle.Transposed(g)
    rng = np.random.default_rng(1)
    ones = np.ones(g.m, dtype=np.uint8)
    picks = np.concatenate([rng.integers(0, g.m, size=20), [int(np.argmax(theta))],
                            rng.choice(np.nonzero(theta > np.median(theta))[0], size=4)])
    for e in picks:
        e = int(e)
        th = int(theta[e])
        assert t.edge_support_within(ones, e) == int(ce[e])
        if th > 0:
            assert t.edge_support_within(theta >= th, e) >= th
        assert t.edge_support_within(theta >= th + 1, e) <= th
