"""Seeded synthetic bipartite graph inputs, shared by the oracle and the GPU path.

This package draws graphs only; it contains none of the counting or peeling
arithmetic.  Graphs are returned as a U-side CSR: ``u_off`` (uint64, nu+1)
and ``u_adj`` (uint32, m), rows sorted ascending, no duplicates.  The edge id
of an edge is its position in ``u_adj``.

Workload recipes (stand-ins for the paper's KONECT graphs, Sec. 6.1 Tab. 2):
uniform random bipartite graphs, Chung-Lu power-law graphs with a degree cap,
and Chung-Lu graphs with planted dense bicliques.  ``CONFIGS`` holds the five
benchmark workloads plus scaled-down variants the oracle finishes quickly.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libbigraph_gen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libbigraph_gen.so (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.gen_uniform.restype = ctypes.c_int64
        lib.gen_uniform.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, P, P]
        lib.gen_chung_lu.restype = ctypes.c_int64
        lib.gen_chung_lu.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, P, P]
        lib.gen_batch_shape.restype = None
        lib.gen_batch_shape.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint32,
                                        ctypes.c_uint32, P, ctypes.POINTER(ctypes.c_double)]
        lib.gen_det_pow.restype = ctypes.c_double
        lib.gen_det_pow.argtypes = [ctypes.c_double, ctypes.c_double]
        _lib = lib
    return _lib


@dataclass
class Graph:
    """A bipartite graph as a U-side CSR (host numpy arrays)."""
    nu: int
    nv: int
    u_off: np.ndarray  # uint64[nu+1]
    u_adj: np.ndarray  # uint32[m]

    @property
    def m(self) -> int:
        return int(self.u_adj.shape[0])

    def edges(self):
        """(eu, ev) arrays in edge-id order."""
        eu = np.repeat(np.arange(self.nu, dtype=np.uint32), np.diff(self.u_off).astype(np.int64))
        return eu, self.u_adj.copy()

    def swapped(self) -> "Graph":
        """The same graph with the roles of U and V exchanged (V-side CSR)."""
        eu, ev = self.edges()
        return from_edges(self.nv, self.nu, ev, eu)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def from_edges(nu: int, nv: int, eu, ev) -> Graph:
    """Build a sorted, de-duplicated U-CSR from edge lists."""
    eu = np.asarray(eu, dtype=np.uint64)
    ev = np.asarray(ev, dtype=np.uint64)
    key = np.unique((eu << np.uint64(32)) | ev)
    u = (key >> np.uint64(32)).astype(np.int64)
    v = (key & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    off = np.zeros(nu + 1, dtype=np.uint64)
    np.add.at(off, u + 1, 1)
    off = np.cumsum(off, dtype=np.uint64)
    return Graph(int(nu), int(nv), off, v)


def uniform(nu: int, nv: int, m: int, seed: int) -> Graph:
    """m distinct (u, v) pairs drawn uniformly at random."""
    off = np.zeros(nu + 1, dtype=np.uint64)
    adj = np.zeros(max(m, 1), dtype=np.uint32)
    rc = _get().gen_uniform(nu, nv, m, seed, _ptr(off), _ptr(adj))
    if rc < 0:
        raise ValueError(f"gen_uniform failed ({rc})")
    return Graph(nu, nv, off, adj[:rc])


def chung_lu(nu: int, nv: int, m: int, gamma_u: float, gamma_v: float, dmax: int, seed: int,
             nplant: int = 0, plant_lo: int = 0, plant_hi: int = 0) -> Graph:
    """Chung-Lu power-law bipartite graph (+ optional planted bicliques)."""
    cap = m + nplant * plant_hi * plant_hi
    off = np.zeros(nu + 1, dtype=np.uint64)
    adj = np.zeros(max(cap, 1), dtype=np.uint32)
    rc = _get().gen_chung_lu(nu, nv, m, gamma_u, gamma_v, dmax, nplant, plant_lo, plant_hi, seed, cap,
                             _ptr(off), _ptr(adj))
    if rc < 0:
        raise ValueError(f"gen_chung_lu failed ({rc})")
    return Graph(nu, nv, off, adj[:rc].copy())


def complete(a: int, b: int) -> Graph:
    """K_{a,b}."""
    eu = np.repeat(np.arange(a), b)
    ev = np.tile(np.arange(b), a)
    return from_edges(a, b, eu, ev)


def batch_shape(seed: int, m_lo=1000, m_hi=200000, r_lo=1.0, r_hi=8.0, g_lo=2.0, g_hi=2.8,
                plant_max=5, dmax_cap=50000):
    out = np.zeros(5, dtype=np.uint64)
    g = ctypes.c_double()
    _get().gen_batch_shape(seed, m_lo, m_hi, r_lo, r_hi, g_lo, g_hi, plant_max, dmax_cap, _ptr(out),
                           ctypes.byref(g))
    m, nu, nv, nplant, dmax = (int(x) for x in out)
    return dict(m=m, nu=nu, nv=nv, nplant=nplant, dmax=dmax, gamma=float(g.value))


def batch_graph(seed: int, scale: float = 1.0, **kw) -> Graph:
    """One graph of the heterogeneous batch workload (seeded by ``seed``).

    ``scale`` shrinks the edge-count range (used by the reduced test variant)."""
    kw.setdefault("m_lo", max(200, int(1000 * scale)))
    kw.setdefault("m_hi", max(400, int(200000 * scale)))
    s = batch_shape(seed, **kw)
    return chung_lu(s["nu"], s["nv"], s["m"], s["gamma"], s["gamma"], s["dmax"], seed,
                    nplant=s["nplant"], plant_lo=5, plant_hi=50 if scale >= 1.0 else 12)


def det_pow(x: float, a: float) -> float:
    return float(_get().gen_det_pow(x, a))


# --------------------------------------------------------------------------
# Workloads.  Each entry: (kind, params).  Full-size entries are the five
# benchmark configurations; *_small entries are the same recipe scaled down
# so the oracle finishes in seconds while still spanning many GPU tiles.
CONFIGS = {
    # uniform |U|=2000 |V|=1000 m=20000, tip of U, P=8
    "uniform_2k_1k_20k": dict(kind="uniform", nu=2000, nv=1000, m=20000, seed=1),
    # Chung-Lu |U|=1M |V|=200k m=20M, exponents 2.1 / 2.5, degree cap 50k; tip of both sides, P=150
    "chunglu_1m_200k_20m": dict(kind="chung_lu", nu=1000000, nv=200000, m=20000000, gu=2.1, gv=2.5,
                                dmax=50000, seed=2),
    # Chung-Lu |U|=500k |V|=100k m=5M, exponents 2.2 / 2.4 + 200 planted 20..200 bicliques; wing, P=100
    "chunglu_500k_100k_5m_planted": dict(kind="chung_lu", nu=500000, nv=100000, m=5000000, gu=2.2, gv=2.4,
                                         dmax=50000, seed=3, nplant=200, plant_lo=20, plant_hi=200),
    # the same planted recipe on a 1M-edge Chung-Lu base (all 200 bicliques kept): the
    # oracle's wing peeling finishes it in under an hour
    "chunglu_500k_100k_1m_planted": dict(kind="chung_lu", nu=500000, nv=100000, m=1000000, gu=2.2, gv=2.4,
                                         dmax=50000, seed=3, nplant=200, plant_lo=20, plant_hi=200),
    # Chung-Lu |U|=5M |V|=1M m=60M, exponents 2.1 / 2.3; tip of U, P=200
    "chunglu_5m_1m_60m": dict(kind="chung_lu", nu=5000000, nv=1000000, m=60000000, gu=2.1, gv=2.3,
                              dmax=50000, seed=5),
    # reduced variants of the same recipes
    "chunglu_20k_4k_200k": dict(kind="chung_lu", nu=20000, nv=4000, m=200000, gu=2.1, gv=2.5, dmax=2000,
                                seed=12),
    "chunglu_5k_1k_50k_planted": dict(kind="chung_lu", nu=5000, nv=1000, m=50000, gu=2.2, gv=2.4, dmax=1000,
                                      seed=13, nplant=6, plant_lo=8, plant_hi=30),
}


def make(name_or_spec) -> Graph:
    """Generate a named workload (see ``CONFIGS``) or an explicit spec dict."""
    spec = dict(CONFIGS[name_or_spec]) if isinstance(name_or_spec, str) else dict(name_or_spec)
    kind = spec.pop("kind") if "kind" in spec else "chung_lu"
    if kind == "uniform":
        return uniform(spec["nu"], spec["nv"], spec["m"], spec["seed"])
    return chung_lu(spec["nu"], spec["nv"], spec["m"], spec["gu"], spec["gv"], spec["dmax"], spec["seed"],
                    spec.get("nplant", 0), spec.get("plant_lo", 0), spec.get("plant_hi", 0))
