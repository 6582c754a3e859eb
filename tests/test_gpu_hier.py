"""k-tips from tip numbers: the CUDA library against the oracle (same tip
numbers in, identical component labels out), warp and block classes."""
import numpy as np
import pytest

import bigraph_gen as gen
import oracle
from oracle import hier

pytestmark = pytest.mark.gpu
pytest.importorskip("scipy")


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


def graphs():
    rng = np.random.default_rng(3)
    a = rng.random((40, 30)) < 0.3
    eu, ev = np.nonzero(a)
    return {
        "rand_40_30": gen.from_edges(40, 30, eu, ev),
        "uniform_2k_1k_20k": gen.make("uniform_2k_1k_20k"),
        "chunglu_5k_1k_50k_planted": gen.make("chunglu_5k_1k_50k_planted"),
        "chunglu_20k_4k_200k": gen.make("chunglu_20k_4k_200k"),
    }


GRAPHS = graphs()


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("side", ["U", "V"])
def test_components_match_oracle(pbng, name, side):
    import torch
    g = GRAPHS[name]
    theta = oracle.tip(g, side)
    dg = pbng.to_device(g)
    th = torch.as_tensor(theta.view(np.int64), device="cuda")
    levels = np.unique(theta)
    ks = sorted({0, 1, int(levels[len(levels) // 2]), int(levels[-1]), int(levels[-1]) + 1,
                 int(levels[max(0, len(levels) // 4)])})
    for k in ks:
        got, st = pbng.tip_components(dg, side, th, k, with_stats=True)
        got = got.cpu().numpy().view(np.uint32)
        want = hier.tip_components(g, side, theta, k)
        assert np.array_equal(got, want), (name, side, k)


def test_components_heavy_members(pbng):
    """Members with many wedges (block class, dense counters in global memory)."""
    import torch
    rng = np.random.default_rng(91)
    nu, nv = 20000, 300
    eu = [np.arange(nu)] + [np.arange(0, 6000)] * 2
    ev = [rng.integers(3, nv, size=nu), np.zeros(6000, np.int64), np.ones(6000, np.int64)]
    key = np.unique(np.concatenate(eu).astype(np.int64) * nv + np.concatenate(ev))
    g = gen.from_edges(nu, nv, key // nv, key % nv)
    theta = oracle.tip(g, "U")
    dg = pbng.to_device(g)
    th = torch.as_tensor(theta.view(np.int64), device="cuda")
    for k in (1, int(theta.max()) // 2, int(theta.max())):
        got = pbng.tip_components(dg, "U", th, k).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, hier.tip_components(g, "U", theta, k)), k


@pytest.mark.parametrize("name", ["rand_40_30", "uniform_2k_1k_20k", "chunglu_5k_1k_50k_planted"])
def test_wing_components_match_oracle(pbng, name):
    import torch
    g = GRAPHS[name]
    theta = oracle.wing(g)
    dg = pbng.to_device(g)
    th = torch.as_tensor(theta.view(np.int64), device="cuda")
    levels = np.unique(theta)
    for k in sorted({0, 1, int(levels[len(levels) // 2]), int(levels[-1]), int(levels[-1]) + 1}):
        got = pbng.wing_components(dg, th, k).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, hier.wing_components(g, theta, k)), (name, k)


def test_wing_components_heavy_vertex(pbng):
    """A U vertex adjacent to every V vertex (block class)."""
    import torch
    rng = np.random.default_rng(8)
    nu, nv = 400, 600
    eu = [np.zeros(nv, np.int64), rng.integers(1, nu, size=2000)]
    ev = [np.arange(nv), rng.integers(0, nv, size=2000)]
    key = np.unique(np.concatenate(eu) * nv + np.concatenate(ev))
    g = gen.from_edges(nu, nv, key // nv, key % nv)
    theta = oracle.wing(g)
    dg = pbng.to_device(g)
    th = torch.as_tensor(theta.view(np.int64), device="cuda")
    for k in (1, int(np.median(theta)), int(theta.max())):
        got = pbng.wing_components(dg, th, k).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, hier.wing_components(g, theta, k)), k
