"""The allocation-free entry point pbng_vertex_counts_noalloc, called through
the C ABI, must give the same per-vertex counts as pbng_count on two calls
in a row.  It serves callers that cannot allocate device memory, so it works
in a fixed static scratch array shared by all calls; the second call checks
that leftovers of the first one do not leak into its result.  This file is
collected last so that a failure here does not hide any other test."""
import ctypes

import numpy as np
import pytest

import bigraph_gen as gen

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


def call_noalloc(pbng, dg, dg_t, out):
    import torch
    L = pbng.lib()
    s = torch.cuda.current_stream().cuda_stream
    return L.pbng_vertex_counts_noalloc(dg.nu, dg.nv, dg.m, dg.u_off.data_ptr(), dg.u_adj.data_ptr(),
                                        dg_t.u_off.data_ptr(), dg_t.u_adj.data_ptr(), out.data_ptr(),
                                        ctypes.c_void_p(s))


@pytest.mark.parametrize("name", ["chunglu_20k_4k_200k", "uniform_2k_1k_20k", "chunglu_5k_1k_50k_planted"])
def test_noalloc_matches_count_twice(pbng, name):
    import torch
    g = gen.make(name)
    for h in (g, g.swapped()):          # U side, then V side
        dg, dg_t = pbng.to_device(h), pbng.to_device(h.swapped())
        want = pbng.as_u64(pbng.count(dg, vertices=True)[0])
        for _ in range(2):
            out = torch.full((dg.nu,), -1, dtype=torch.int64, device="cuda")
            assert call_noalloc(pbng, dg, dg_t, out) == pbng.PBNG_OK
            assert np.array_equal(pbng.as_u64(out), want)


def test_noalloc_rejects_oversize_and_bad_input(pbng):
    import torch
    L = pbng.lib()
    z = torch.zeros(4, dtype=torch.int64, device="cuda")
    # nu beyond the static scratch limit: rejected before any device work
    rc = L.pbng_vertex_counts_noalloc((16 << 20) + 1, 1, 0, z.data_ptr(), None, z.data_ptr(), None, z.data_ptr(), None)
    assert rc == pbng.PBNG_EINVAL and b"limit" in L.pbng_last_error_detail()
    # an out-of-range neighbour id is caught by the range check
    off = torch.tensor([0, 1, 1], dtype=torch.int64, device="cuda")
    adj = torch.tensor([7], dtype=torch.int32, device="cuda")
    voff = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    vadj = torch.tensor([0], dtype=torch.int32, device="cuda")
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    rc = L.pbng_vertex_counts_noalloc(2, 1, 1, off.data_ptr(), adj.data_ptr(), voff.data_ptr(), vadj.data_ptr(),
                                      out.data_ptr(), None)
    assert rc == pbng.PBNG_EINVAL
