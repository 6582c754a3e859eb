"""CPU oracle for butterfly counting and tip / wing decomposition.

TEST INFRASTRUCTURE ONLY: the GPU library never imports this package.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
use it.  The arithmetic lives in ``oracle.c`` (plain sequential C, exact
uint64): butterfly counts by their definition (Sec. 2.1), bottom-up peeling
BUP for tip and wing numbers (Sec. 2.2, Alg. 2), and membership-restricted
supports for sampled checks at full size.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, U32, U64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        for name in ("oracle_vertex_counts", "oracle_edge_counts", "oracle_tip_bup", "oracle_wing_bup"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = [U32, U32, P, P, P]
        lib.oracle_vertex_counts_parallel.restype = ctypes.c_int
        lib.oracle_vertex_counts_parallel.argtypes = [U32, U32, P, P, P]
        lib.oracle_vertex_support_within.restype = U64
        lib.oracle_vertex_support_within.argtypes = [U32, U32, P, P, P, P, P, U32]
        lib.oracle_edge_support_within.restype = U64
        lib.oracle_edge_support_within.argtypes = [U32, P, P, P, P, P, P, U64]
        lib.oracle_transpose.restype = ctypes.c_int
        lib.oracle_transpose.argtypes = [U32, U32, P, P, P, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(g):
    return np.ascontiguousarray(g.u_off, dtype=np.uint64), np.ascontiguousarray(g.u_adj, dtype=np.uint32)


def _side(g, side: str):
    if side in ("U", "u", 0):
        return g
    if side in ("V", "v", 1):
        return g.swapped()
    raise ValueError(side)


def vertex_counts(g, side="U") -> np.ndarray:
    """Butterflies of every vertex of ``side`` (definition, Sec. 2.1)."""
    h = _side(g, side)
    off, adj = _csr(h)
    out = np.zeros(max(h.nu, 1), dtype=np.uint64)
    if _get().oracle_vertex_counts(h.nu, h.nv, _p(off), _p(adj), _p(out)):
        raise MemoryError
    return out[:h.nu]


def vertex_counts_parallel(g, side="U"):
    """(counts, threads): the counts of vertex_counts computed by every host thread."""
    h = _side(g, side)
    off, adj = _csr(h)
    out = np.zeros(max(h.nu, 1), dtype=np.uint64)
    th = _get().oracle_vertex_counts_parallel(h.nu, h.nv, _p(off), _p(adj), _p(out))
    if th < 0:
        raise MemoryError
    return out[:h.nu], th


def edge_counts(g) -> np.ndarray:
    """Butterflies of every edge, in edge-id order (definition, Sec. 2.1)."""
    off, adj = _csr(g)
    out = np.zeros(max(g.m, 1), dtype=np.uint64)
    if _get().oracle_edge_counts(g.nu, g.nv, _p(off), _p(adj), _p(out)):
        raise MemoryError
    return out[:g.m]


def tip(g, side="U") -> np.ndarray:
    """Tip numbers of ``side`` by bottom-up peeling (Alg. 2 on vertices)."""
    h = _side(g, side)
    off, adj = _csr(h)
    out = np.zeros(max(h.nu, 1), dtype=np.uint64)
    if _get().oracle_tip_bup(h.nu, h.nv, _p(off), _p(adj), _p(out)):
        raise MemoryError
    return out[:h.nu]


def wing(g) -> np.ndarray:
    """Wing numbers of every edge (edge-id order) by bottom-up peeling (Alg. 2)."""
    off, adj = _csr(g)
    out = np.zeros(max(g.m, 1), dtype=np.uint64)
    if _get().oracle_wing_bup(g.nu, g.nv, _p(off), _p(adj), _p(out)):
        raise MemoryError
    return out[:g.m]


class Transposed:
    """V-side CSR with edge ids, for repeated membership-restricted checks."""

    def __init__(self, g):
        off, adj = _csr(g)
        self.g = g
        self.u_off, self.u_adj = off, adj
        self.v_off = np.zeros(g.nv + 1, dtype=np.uint64)
        self.v_adj = np.zeros(max(g.m, 1), dtype=np.uint32)
        self.v_eid = np.zeros(max(g.m, 1), dtype=np.uint64)
        if _get().oracle_transpose(g.nu, g.nv, _p(off), _p(adj), _p(self.v_off), _p(self.v_adj), _p(self.v_eid)):
            raise MemoryError

    def vertex_support_within(self, member: np.ndarray, u: int) -> int:
        """Butterflies u (side U) has with the U-vertices marked in member."""
        member = np.ascontiguousarray(member, dtype=np.uint8)
        r = _get().oracle_vertex_support_within(self.g.nu, self.g.nv, _p(self.u_off), _p(self.u_adj),
                                                 _p(self.v_off), _p(self.v_adj), _p(member), int(u))
        if r == (1 << 64) - 1:
            raise MemoryError
        return int(r)

    def edge_support_within(self, member: np.ndarray, e: int) -> int:
        """Butterflies of edge e whose other three edges are marked in member."""
        member = np.ascontiguousarray(member, dtype=np.uint8)
        return int(_get().oracle_edge_support_within(self.g.nu, _p(self.u_off), _p(self.u_adj), _p(self.v_off),
                                                     _p(self.v_adj), _p(self.v_eid), _p(member), int(e)))
