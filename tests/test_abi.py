"""The C-ABI library loads, exports every entry point declared in
include/pbng.h, has struct layouts that match the header, and rejects
invalid arguments on the host before touching the GPU (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pbng.h")


@pytest.fixture(scope="module")
def L():
    from paper_2110_12511_gb300 import build as b
    b.build()
    import paper_2110_12511_gb300 as pbng
    return pbng.lib()


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(pbng_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 8
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2110_12511_gb300", "libpbng.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (pbng_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(L, n)


def test_struct_layout_matches_header(tmp_path):
    import paper_2110_12511_gb300 as pbng
    src = tmp_path / "sz.c"
    src.write_text('#include "pbng.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(){printf("%zu %zu %zu %zu %zu %zu\\n",'
                   'sizeof(pbng_bigraph),sizeof(pbng_opts),sizeof(pbng_stats),offsetof(pbng_opts,stream),'
                   'offsetof(pbng_stats,parts_used),offsetof(pbng_opts,learned_vet));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(pbng.Bigraph), ctypes.sizeof(pbng.Opts), ctypes.sizeof(pbng.Stats),
            pbng.Opts.stream.offset, pbng.Stats.parts_used.offset, pbng.Opts.learned_vet.offset]
    assert got == want


def test_host_side_argument_checks(L):
    import paper_2110_12511_gb300 as pbng
    off = np.zeros(3, dtype=np.uint64)
    g = pbng.Bigraph(2, 2, 0, off.ctypes.data, 0)
    out = np.zeros(2, dtype=np.uint64)
    o = pbng.Opts()
    L.pbng_opts_init(ctypes.byref(o))
    assert o.recount == 1 and o.compact == 1 and o.bounds_mode == 0
    # P = 0
    assert L.pbng_tip_decompose(ctypes.byref(g), 0, 0, out.ctypes.data, ctypes.byref(o), None) == pbng.PBNG_EINVAL
    # bad side
    assert L.pbng_tip_decompose(ctypes.byref(g), 7, 4, out.ctypes.data, ctypes.byref(o), None) == pbng.PBNG_EINVAL
    # null output
    assert L.pbng_tip_decompose(ctypes.byref(g), 0, 4, None, ctypes.byref(o), None) == pbng.PBNG_EINVAL
    # explicit bounds that are not strictly increasing
    b = np.array([5, 5, 9], dtype=np.uint64)
    o.bounds_mode = pbng.BOUNDS_EXPLICIT
    o.bounds = b.ctypes.data
    o.n_bounds = 3
    assert L.pbng_tip_decompose(ctypes.byref(g), 0, 4, out.ctypes.data, ctypes.byref(o), None) == pbng.PBNG_EBOUNDS
    assert b"increasing" in L.pbng_last_error_detail()
    # a NaN learned-bound judge
    o.bounds_mode = 0
    o.learned_vet = float("nan")
    assert L.pbng_tip_decompose(ctypes.byref(g), 0, 4, out.ctypes.data, ctypes.byref(o), None) == pbng.PBNG_EINVAL
    assert b"learned_vet" in L.pbng_last_error_detail()
    o.learned_vet = 0.0
    # oversize graph
    big = pbng.Bigraph(1 << 30, 1 << 30, 0, off.ctypes.data, 0)
    o.bounds_mode = 0
    assert L.pbng_count(ctypes.byref(big), None, None, None, ctypes.byref(o), None) == pbng.PBNG_EINVAL
    assert L.pbng_strerror(pbng.PBNG_EBOUNDS) == b"bounds not strictly increasing"
    assert L.pbng_version() >= 100
