"""Host-side logic that needs no GPU: the learned proposer's target encoding
and candidate bounds, and the autotuner's graph signature."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2110_12511_gb300 import autotune as at
from paper_2110_12511_gb300 import learned


def test_encode_decode_round_trip():
    K = 10 ** 9
    b = np.array([3, 17, 1000, 123456, 10 ** 8], dtype=np.uint64)
    y = learned.encode(b, 8, K)
    assert y.shape == (8,) and (np.diff(y) >= 0).all()
    d = learned.decode(y[:5], K)
    assert (np.abs(d.astype(np.float64) - b.astype(np.float64)) <= 1e-3 * b.astype(np.float64) + 1).all()
    assert (np.diff(learned.decode(y, K).astype(np.float64)) > 0).all()  # strictly increasing after decoding


def test_quantile_bounds_split_work_evenly():
    rng = np.random.default_rng(0)
    theta = rng.integers(0, 10 ** 6, size=5000).astype(np.float64)
    work = rng.integers(1, 100, size=5000).astype(np.float64)
    P = 10
    b = learned.quantile_bounds(theta, work, P).astype(np.float64)
    assert (np.diff(b) > 0).all() and len(b) <= P - 1
    edges = np.concatenate([[-1], b, [np.inf]])
    parts = [work[(theta >= lo) & (theta < hi)].sum() for lo, hi in zip(edges[:-1], edges[1:])]
    assert max(parts) <= 2.0 * work.sum() / P + work.max()


def test_blend_interpolates_in_log_space():
    a = np.array([10, 100, 1000], dtype=np.uint64)
    b = np.array([1000, 10000, 100000], dtype=np.uint64)
    m = learned.blend(a, b, 0.5, 4).astype(np.float64)
    assert (np.diff(m) > 0).all()
    assert np.allclose(np.log2(1 + m), 0.5 * (np.log2(1 + a) + np.log2(1 + b)), atol=0.05)


def test_signature_depends_on_sizes_and_degrees():
    class G:
        def __init__(self, off, nv):
            self.u_off = torch.as_tensor(np.asarray(off, dtype=np.int64))
            self.nu = len(off) - 1
            self.nv = nv
            self.m = int(off[-1])

    g1 = G([0, 2, 4, 8], 5)
    g2 = G([0, 1, 4, 8], 5)
    assert at.signature(g1, "U", 10) != at.signature(g2, "U", 10)  # different degree histograms
    assert at.signature(g1, "U", 10) != at.signature(g1, "V", 10)
    assert at.signature(g1, "U", 10) != at.signature(g1, "U", 20)
    assert at.signature(g1, "U", 10) == at.signature(G([0, 2, 4, 8], 5), "U", 10)


def test_candidates_cover_estimator_quantiles_and_blends():
    est = np.array([5, 50, 500], dtype=np.uint64)
    wq = np.array([20, 2000, 20000], dtype=np.uint64)
    c = learned.candidates(est, wq, 4)
    assert set(c) == {"estimator", "work_quantiles", "blend_0.25", "blend_0.5", "blend_0.75"}
    # blends move monotonically from the estimator's bounds towards the quantiles
    logs = [np.log2(1 + c[k].astype(np.float64)).mean() for k in ("blend_0.25", "blend_0.5", "blend_0.75")]
    assert logs[0] < logs[1] < logs[2]


def test_training_recipes_are_seeded_and_in_range():
    from paper_2110_12511_gb300 import train_bounds as tb
    g1 = tb.training_wing_graph(3, 20000, 40000)
    g2 = tb.training_wing_graph(3, 20000, 40000)
    assert np.array_equal(g1.u_off, g2.u_off) and np.array_equal(g1.u_adj, g2.u_adj)
    # base edges in range, plus at most 200 planted bicliques of up to 200 x 200
    assert 20000 * 0.9 <= g1.m <= 40000 + 200 * 200 * 200
    assert g1.nu >= 2000 and g1.nv >= 400
    t = tb.training_graph(1, 20000, 40000)
    assert 10000 <= t.m <= 40000 and t.nu + t.nv <= 4000 + 2
