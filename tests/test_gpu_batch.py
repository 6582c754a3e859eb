"""GPU checks of the batch calls: every graph's own CSR is validated before
the disjoint union is formed (a bad id or offset would otherwise move edges
into a neighbouring graph), host-memory batches match the oracle, and the
bounds used are reported."""
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


class RawGraph:
    """A CSR taken as given (no sorting or de-duplication)."""

    def __init__(self, nu, nv, off, adj):
        self.nu, self.nv = nu, nv
        self.u_off = np.asarray(off, dtype=np.uint64)
        self.u_adj = np.asarray(adj, dtype=np.uint32)

    @property
    def m(self):
        return int(self.u_adj.size)


def good_graphs():
    return [gen.complete(3, 4), gen.make("chunglu_5k_1k_50k_planted"), gen.complete(2, 2)]


BAD = {
    # graph index 0: a neighbour id equal to its own nv (valid in the union, where it
    # would name the next graph's first V vertex)
    "id_equals_nv": (0, RawGraph(2, 3, [0, 2, 3], [0, 3, 1])),
    # graph index 1: first offset not zero
    "offset0_nonzero": (1, RawGraph(2, 2, [1, 2, 3], [0, 1, 0])),
    # graph index 2: last offset differs from m
    "last_offset": (2, RawGraph(2, 2, [0, 1, 2], [0, 1, 1])),
    # graph index 1: a row that is not strictly increasing
    "unsorted_row": (1, RawGraph(2, 3, [0, 2, 3], [2, 1, 0])),
}


def with_bad(idx, bad):
    gs = good_graphs()
    gs.insert(idx, bad)
    return gs


@pytest.mark.parametrize("case", list(BAD))
@pytest.mark.parametrize("kind", ["tip", "wing"])
def test_batch_rejects_a_malformed_graph(pbng, case, kind):
    idx, bad = BAD[case]
    gs = with_bad(idx, bad)
    dgs = [pbng.to_device(g) for g in gs]
    with pytest.raises(pbng.PbngError) as ei:
        if kind == "tip":
            pbng.tip_decompose_batch(dgs, "U", P=8)
        else:
            pbng.wing_decompose_batch(dgs, P=8)
    assert ei.value.code == pbng.PBNG_EINVAL
    assert f"graph {idx}" in str(ei.value)
    # host-memory batches run the same check
    with pytest.raises(pbng.PbngError) as ei:
        if kind == "tip":
            pbng.tip_decompose_batch_host(gs, "U", P=8)
        else:
            pbng.wing_decompose_batch_host(gs, P=8)
    assert ei.value.code == pbng.PBNG_EINVAL and f"graph {idx}" in str(ei.value)


def used_count(bo, st):
    """Bounds written: one per range closed by a finite bound (parts_used - 1,
    or parts_used when a finite bound took every remaining entity)."""
    k = int(np.count_nonzero(bo))
    assert k in (st["parts_used"] - 1, st["parts_used"]) and not bo[k:].any()
    return k


def batch_graphs():
    gs = [gen.batch_graph(3000 + i, scale=0.02) for i in range(6)]
    gs.insert(2, gen.from_edges(3, 2, [], []))  # edgeless: NULL output for wing
    gs.append(gen.make("chunglu_5k_1k_50k_planted"))
    return gs


@pytest.mark.parametrize("side", ["U", "V"])
def test_tip_batch_host_memory_matches_oracle(pbng, side):
    gs = batch_graphs()
    bo = np.zeros(64, dtype=np.uint64)
    got, st = pbng.tip_decompose_batch_host(gs, side, P=20, with_stats=True, bounds_out=bo)
    for g, t in zip(gs, got):
        assert np.array_equal(t, oracle.tip(g, side))
    k = used_count(bo, st)
    assert k >= 1 and np.all(np.diff(bo[:k].astype(np.float64)) > 0)
    assert st["ns_setup"] > 0


def test_wing_batch_host_memory_matches_oracle(pbng):
    gs = batch_graphs()
    bo = np.zeros(64, dtype=np.uint64)
    got, st = pbng.wing_decompose_batch_host(gs, P=20, with_stats=True, bounds_out=bo)
    for g, w in zip(gs, got):
        assert np.array_equal(w, oracle.wing(g))
    k = used_count(bo, st)
    assert k >= 1 and np.all(np.diff(bo[:k].astype(np.float64)) > 0)
    assert st["ns_setup"] > 0
    # the device-memory batch agrees and reports the same bounds
    bo2 = np.zeros(64, dtype=np.uint64)
    dev = pbng.wing_decompose_batch([pbng.to_device(g) for g in gs], P=20, bounds_out=bo2)
    for w, d in zip(got, dev):
        assert np.array_equal(w, pbng.as_u64(d))
    assert np.array_equal(bo, bo2)
