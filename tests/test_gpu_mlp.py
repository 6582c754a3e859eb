"""The learned bound proposer's CUDA kernels against the FP64 oracle, and the
learned bounds against the method without them (identical tip numbers)."""
import os

import numpy as np
import pytest

import bigraph_gen as gen
import oracle
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu
DATA = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2110_12511_gb300", "data")
WEIGHTS = os.path.join(DATA, "bound_mlp_p200.npz")
WING_WEIGHTS = os.path.join(DATA, "bound_mlp_wing_p100.npz")


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


def rand_problem(seed, dims=(128, 128, 199), B=16):
    from paper_2110_12511_gb300 import learned
    rng = np.random.default_rng(seed)
    p = learned.init_params(dims[2], seed, nin=dims[0], hid=dims[1])
    p = p + rng.normal(0, 0.01, size=learned.n_params(*dims)).astype(np.float32)
    X = rng.random((B, dims[0])).astype(np.float32)
    T = rng.random((B, dims[2])).astype(np.float32)
    return p, X, T


def test_forward_and_gradient_match_fp64_oracle(pbng):
    import torch
    for seed, dims in ((0, (128, 128, 199)), (1, (7, 5, 3))):
        p, X, T = rand_problem(seed, dims, B=16 if dims[0] == 128 else 4)
        pd, Xd, Td = (torch.as_tensor(a, device="cuda") for a in (p, X, T))
        Y = pbng.mlp_forward(pd, dims, Xd).cpu().numpy()
        Yo = omlp.forward(p, dims, X)
        assert np.allclose(Y, Yo, rtol=1e-4, atol=1e-5)
        g, loss = pbng.mlp_grad(pd, dims, Xd, Td)
        go, lo = omlp.grad(p, dims, X, T)
        g = g.cpu().numpy().astype(np.float64)
        assert abs(loss - lo) <= 1e-5 * max(1.0, lo)
        assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
        assert np.allclose(g, go, rtol=1e-3, atol=1e-6 * np.abs(go).max())


def test_adam_step_matches_formula(pbng):
    import torch
    rng = np.random.default_rng(3)
    n = 1000
    p, g = rng.normal(size=n).astype(np.float32), rng.normal(size=n).astype(np.float32)
    m, v = rng.normal(size=n).astype(np.float32) * 0.1, np.abs(rng.normal(size=n)).astype(np.float32) * 0.1
    pd, gd, md, vd = (torch.as_tensor(a.copy(), device="cuda") for a in (p, g, m, v))
    pbng.mlp_adam(pd, gd, md, vd, 1e-2, 5)
    b1, b2, eps = 0.9, 0.999, 1e-8
    m2 = b1 * m + (1 - b1) * g
    v2 = b2 * v + (1 - b2) * g * g
    p2 = p - 1e-2 * (m2 / (1 - b1 ** 5)) / (np.sqrt(v2 / (1 - b2 ** 5)) + eps)
    assert np.allclose(pd.cpu().numpy(), p2, rtol=1e-5, atol=1e-6)


def half_octave(d):
    d = np.asarray(d, dtype=np.int64)
    out = d.copy()
    big = d >= 2
    L = np.zeros_like(d)
    L[big] = np.floor(np.log2(d[big])).astype(np.int64) + 1
    out[big] = 2 * L[big] - 2 + ((d[big] >> (L[big] - 2)) & 1)
    return np.minimum(out, 63)


def test_features_match_oracle_counts(pbng):
    g = gen.make("chunglu_5k_1k_50k_planted")
    for side in ("U", "V"):
        h = g if side == "U" else g.swapped()
        f = pbng.bound_features(pbng.to_device(g), side).cpu().numpy()
        cnt = oracle.vertex_counts(g, side)
        deg = np.diff(h.u_off).astype(np.int64)
        fd = np.bincount(half_octave(deg), minlength=64)[:64] / h.nu
        bl = np.array([int(c).bit_length() for c in cnt])
        fs = np.bincount(np.minimum(bl.max() - bl, 63), minlength=64)[:64] / h.nu
        assert np.allclose(f[:64], fd, atol=1e-6) and np.allclose(f[64:], fs, atol=1e-6)


def test_wing_features_match_oracle_counts(pbng):
    """Wing features: min(d_u, d_v) per edge and the oracle's per-edge counts."""
    g = gen.make("chunglu_5k_1k_50k_planted")
    f = pbng.wing_bound_features(pbng.to_device(g)).cpu().numpy()
    du = np.diff(g.u_off).astype(np.int64)
    dv = np.bincount(g.u_adj, minlength=g.nv).astype(np.int64)
    eu = np.repeat(np.arange(g.nu), du)
    deg = np.minimum(du[eu], dv[g.u_adj])
    cnt = oracle.edge_counts(g)
    fd = np.bincount(half_octave(deg), minlength=64)[:64] / g.m
    bl = np.array([int(c).bit_length() for c in cnt])
    fs = np.bincount(np.minimum(bl.max() - bl, 63), minlength=64)[:64] / g.m
    assert np.allclose(f[:64], fd, atol=1e-6) and np.allclose(f[64:], fs, atol=1e-6)


def wing_mlp():
    import torch
    from paper_2110_12511_gb300 import learned
    if os.path.exists(WING_WEIGHTS):
        return learned.load(WING_WEIGHTS)
    return torch.as_tensor(learned.init_params(99, 2), device="cuda"), 128, 99


@pytest.mark.parametrize("vet", [0.0, -1.0])
@pytest.mark.parametrize("name", ["chunglu_5k_1k_50k_planted", "rand_dense"])
def test_learned_wing_bounds_give_identical_wing_numbers(pbng, name, vet):
    """Learned wing bounds, judged by the estimator or not: the oracle's wing
    numbers (Th. 2), and the bounds reported are strictly increasing."""
    g = gen.make(name) if name != "rand_dense" else gen.uniform(60, 50, 1500, 9)
    dg = pbng.to_device(g)
    used = np.zeros(100, dtype=np.uint64)
    th, st = pbng.wing_decompose(dg, P=100, mlp=wing_mlp(), learned_vet=vet, with_stats=True, bounds_out=used)
    assert np.array_equal(pbng.as_u64(th), oracle.wing(g))
    b = used[:np.count_nonzero(used)]
    assert b.size in (st["parts_used"] - 1, st["parts_used"])
    assert (np.diff(b.astype(np.float64)) > 0).all()


def test_training_reduces_loss(pbng):
    from paper_2110_12511_gb300 import learned
    rng = np.random.default_rng(4)
    X = rng.random((24, 128)).astype(np.float32)
    W = rng.normal(size=(128, 199)).astype(np.float32) * 0.02
    T = (0.3 + X @ W).astype(np.float32)
    _, losses = learned.train(X, T, 199, epochs=300, lr=2e-3)
    assert losses[-1] < 0.1 * losses[0]


@pytest.mark.parametrize("name", ["chunglu_20k_4k_200k", "chunglu_5k_1k_50k_planted", "uniform_2k_1k_20k"])
def test_learned_bounds_give_identical_tip_numbers(pbng, name):
    import torch
    from paper_2110_12511_gb300 import learned
    g = gen.make(name)
    dg = pbng.to_device(g)
    if os.path.exists(WEIGHTS):
        mlp = learned.load(WEIGHTS)
    else:
        mlp = (torch.as_tensor(learned.init_params(199, 1), device="cuda"), 128, 199)
    used = np.zeros(200, dtype=np.uint64)
    th, st = pbng.tip_decompose(dg, "U", P=200, mlp=mlp, with_stats=True, bounds_out=used)
    assert np.array_equal(pbng.as_u64(th), oracle.tip(g, "U"))
    b = used[:np.count_nonzero(used)]
    assert b.size in (st["parts_used"] - 1, st["parts_used"])
    assert (np.diff(b.astype(np.float64)) > 0).all()


@pytest.mark.parametrize("vet", [-1.0, 0.5, 4.0])
def test_learned_judge_setting_gives_identical_tip_numbers(pbng, vet):
    """Learned bounds unjudged (negative learned_vet), judged strictly and
    loosely: the tip numbers are the oracle's in every case (Th. 2)."""
    import torch
    from paper_2110_12511_gb300 import learned
    g = gen.make("chunglu_20k_4k_200k")
    dg = pbng.to_device(g)
    mlp = learned.load(WEIGHTS) if os.path.exists(WEIGHTS) else (
        torch.as_tensor(learned.init_params(199, 1), device="cuda"), 128, 199)
    th = pbng.tip_decompose(dg, "U", P=200, mlp=mlp, learned_vet=vet)
    assert np.array_equal(pbng.as_u64(th), oracle.tip(g, "U"))


def test_propose_bounds_learned(pbng):
    """pbng_propose_bounds with the learned proposer: the bounds the coarse
    phase uses (learned proposals judged by the estimator) reproduce the
    oracle's tip numbers when passed back explicitly."""
    import torch
    from paper_2110_12511_gb300 import learned
    g = gen.make("chunglu_20k_4k_200k")
    dg = pbng.to_device(g)
    mlp = learned.load(WEIGHTS) if os.path.exists(WEIGHTS) else (
        torch.as_tensor(learned.init_params(199, 1), device="cuda"), 128, 199)
    b = pbng.propose_bounds(dg, "U", P=200, mlp=mlp)
    inner = b[1:][b[1:] != np.iinfo(np.uint64).max]
    used = np.zeros(201, dtype=np.uint64)
    _, st = pbng.tip_decompose(dg, "U", P=200, mlp=mlp, with_stats=True, bounds_out=used)
    assert inner.size in (st["parts_used"] - 1, st["parts_used"])
    assert np.array_equal(used[:inner.size], inner) and not used[inner.size:].any()
    th = pbng.tip_decompose(dg, "U", P=200, bounds=inner)
    assert np.array_equal(pbng.as_u64(th), oracle.tip(g, "U"))


def test_learned_bounds_gain_on_heldout_graph(pbng):
    """What the trained proposer gains over find_range on a graph from its
    training distribution that it never saw (seed 1000): identical tip
    numbers and not slower.  (The estimator vets every learned bound and
    replaces one whose range would hold more than twice its target work.)"""
    import time
    import torch
    from paper_2110_12511_gb300 import learned, train_bounds
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained weights")
    mlp = learned.load(WEIGHTS)
    g = train_bounds.training_graph(1000, 1000000, 60000000)
    dg = pbng.to_device(g)
    def run(m):
        best, res = 1e30, None
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = pbng.tip_decompose(dg, "U", P=200, mlp=m, with_stats=True)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        return best, res
    t_est, (th_est, st_est) = run(None)
    t_lrn, (th_lrn, st_lrn) = run(mlp)
    assert np.array_equal(pbng.as_u64(th_est), pbng.as_u64(th_lrn))
    print(f"learned / find_range time: {t_lrn:.4f} / {t_est:.4f} s = {t_est / t_lrn:.2f}x")
    assert t_lrn <= 1.1 * t_est
