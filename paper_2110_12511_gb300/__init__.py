"""Python binding of libpbng.so: GB300 butterfly counting and two-phase
tip / wing decomposition (Lakhotia, Kannan, Prasanna, "Parallel Peeling of
Bipartite Networks for Hierarchical Dense Subgraph Discovery").

This module only marshals arguments: every step of counting and peeling runs
in the library's CUDA kernels.  PyTorch provides device memory and streams.
Graphs are U-side CSRs (``u_off`` uint64[nu+1], ``u_adj`` uint32[m], rows
sorted, no duplicates); results are uint64, returned as int64 torch tensors
holding the same bits (use ``as_u64`` for a numpy uint64 view).

If the compiled library is missing every call raises: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpbng.so")

PBNG_OK, PBNG_EINVAL, PBNG_ENOMEM, PBNG_ECUDA, PBNG_ETIMEOUT, PBNG_EOVERFLOW, PBNG_EBOUNDS = 0, -1, -2, -3, -4, -5, -6
SIDE_U, SIDE_V = 0, 1
BOUNDS_ESTIMATOR, BOUNDS_LEARNED, BOUNDS_EXPLICIT = 0, 1, 2
MEM_DEVICE, MEM_HOST = 0, 1


class Bigraph(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_uint32), ("nv", ctypes.c_uint32), ("m", ctypes.c_uint64),
                ("u_off", ctypes.c_void_p), ("u_adj", ctypes.c_void_p)]


class Opts(ctypes.Structure):
    _fields_ = [("bounds_mode", ctypes.c_int), ("bounds", ctypes.c_void_p), ("n_bounds", ctypes.c_uint32),
                ("recount", ctypes.c_int), ("compact", ctypes.c_int), ("mem", ctypes.c_int),
                ("graph_rounds", ctypes.c_int), ("timeout_ns", ctypes.c_uint64), ("stream", ctypes.c_void_p),
                ("mlp_params", ctypes.c_void_p), ("mlp_hidden", ctypes.c_uint32), ("mlp_out", ctypes.c_uint32),
                ("bounds_out", ctypes.c_void_p), ("n_bounds_out", ctypes.c_uint32),
                ("bucket_shift", ctypes.c_uint32), ("warp_max_w", ctypes.c_uint32),
                ("group_max_w", ctypes.c_uint32), ("item_w", ctypes.c_uint32), ("fd_cluster_min", ctypes.c_uint32),
                ("count_scratch", ctypes.c_uint32), ("learned_vet", ctypes.c_float)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "wedges_count", "wedges_cd", "wedges_fd", "updates", "links", "blooms", "rounds", "recounts", "fd_steps",
        "wedge_bound", "ns_setup", "ns_count", "ns_cd", "ns_part", "ns_fd", "ns_total")] + [
        ("parts_used", ctypes.c_uint32), ("reserved", ctypes.c_uint32)] + [(n, ctypes.c_uint64) for n in (
        "launches", "ns_k_count", "ns_k_peel", "ns_k_fd", "bytes_count", "bytes_peel", "bytes_fd",
        "n_k_count", "n_k_peel", "n_k_fd", "fd_work_max", "fd_work_sum", "fd_part_steps_max", "fd_part_cycles_max")]

    def to_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "reserved"}


class PbngError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = _lib_or_none()
        name = lib.pbng_strerror(code).decode() if lib else str(code)
        detail = lib.pbng_last_error_detail().decode() if lib else ""
        super().__init__(f"{where}: {name} ({code}){': ' + detail if detail else ''}")
        self.code = code


_lib = None


def _lib_or_none():
    return _lib


def lib():
    """Load libpbng.so (built in-tree by ``paper_2110_12511_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2110_12511_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, C = ctypes.c_void_p, ctypes.c_int
        G, O, S = ctypes.POINTER(Bigraph), ctypes.POINTER(Opts), ctypes.POINTER(Stats)
        L.pbng_opts_init.argtypes = [O]
        L.pbng_opts_init.restype = None
        L.pbng_count.argtypes = [G, P, P, P, O, S]
        L.pbng_count.restype = C
        L.pbng_tip_decompose.argtypes = [G, C, ctypes.c_uint32, P, O, S]
        L.pbng_tip_decompose.restype = C
        L.pbng_wing_decompose.argtypes = [G, ctypes.c_uint32, P, O, S]
        L.pbng_wing_decompose.restype = C
        L.pbng_tip_decompose_batch.argtypes = [G, ctypes.c_uint32, C, ctypes.c_uint32, ctypes.POINTER(P), O, S]
        L.pbng_tip_decompose_batch.restype = C
        L.pbng_wing_decompose_batch.argtypes = [G, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(P), O, S]
        L.pbng_wing_decompose_batch.restype = C
        L.pbng_wing_components.argtypes = [G, P, ctypes.c_uint64, P, O, S]
        L.pbng_wing_components.restype = C
        L.pbng_tip_components.argtypes = [G, C, P, ctypes.c_uint64, P, O, S]
        L.pbng_tip_components.restype = C
        L.pbng_strerror.argtypes = [C]
        L.pbng_strerror.restype = ctypes.c_char_p
        L.pbng_last_error_detail.argtypes = []
        L.pbng_last_error_detail.restype = ctypes.c_char_p
        L.pbng_version.argtypes = []
        L.pbng_version.restype = C
        L.pbng_bound_features.argtypes = [G, C, P, O]
        L.pbng_bound_features.restype = C
        L.pbng_wing_bound_features.argtypes = [G, P, O]
        L.pbng_wing_bound_features.restype = C
        L.pbng_mlp_forward.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, P, ctypes.c_uint32, P, P]
        L.pbng_mlp_forward.restype = C
        L.pbng_mlp_grad.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, P, P, ctypes.c_uint32, P, P, P]
        L.pbng_mlp_grad.restype = C
        L.pbng_mlp_adam.argtypes = [P, P, P, P, ctypes.c_uint64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_uint32, P]
        L.pbng_mlp_adam.restype = C
        L.pbng_propose_bounds.argtypes = [G, C, ctypes.c_uint32, P, O]
        L.pbng_propose_bounds.restype = C
        L.pbng_be_index_sums.argtypes = [G, P, P, O, S]
        L.pbng_be_index_sums.restype = C
        L.pbng_vertex_counts_noalloc.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, P, P, P, P, P, P]
        L.pbng_vertex_counts_noalloc.restype = C
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != PBNG_OK:
        raise PbngError(rc, where)


def as_u64(t) -> np.ndarray:
    """numpy uint64 view of a result tensor (int64 storage of uint64 bits)."""
    return t.detach().cpu().numpy().view(np.uint64)


@dataclass
class DeviceGraph:
    """A bipartite graph resident on the GPU (torch tensors)."""
    nu: int
    nv: int
    u_off: "object"  # torch int64 tensor holding uint64 offsets
    u_adj: "object"  # torch int32 tensor holding uint32 ids

    @property
    def m(self) -> int:
        return int(self.u_adj.numel())

    def c_struct(self) -> Bigraph:
        return Bigraph(self.nu, self.nv, self.m, self.u_off.data_ptr(), self.u_adj.data_ptr() if self.m else 0)


def to_device(g, device="cuda") -> DeviceGraph:
    """Copy a host graph (``bigraph_gen.Graph`` or anything with nu, nv,
    u_off, u_adj numpy arrays) to the GPU."""
    import torch
    off = torch.from_numpy(np.ascontiguousarray(g.u_off, dtype=np.uint64).view(np.int64)).to(device)
    adj = torch.from_numpy(np.ascontiguousarray(g.u_adj, dtype=np.uint32).view(np.int32)).to(device)
    return DeviceGraph(int(g.nu), int(g.nv), off, adj)


SCHEDULE_KEYS = ("bucket_shift", "warp_max_w", "group_max_w", "item_w", "fd_cluster_min", "count_scratch")
SCRATCH_AUTO, SCRATCH_HASH, SCRATCH_DENSE, SCRATCH_DENSE32 = 0, 1, 2, 3


def _opts(stream=None, bounds=None, recount=True, compact=True, mem=MEM_DEVICE, graph_rounds=False, keep=None,
          mlp=None, bounds_out=None, bucket_shift=0, schedule=None, learned_vet=0.0):
    o = Opts()
    lib().pbng_opts_init(ctypes.byref(o))
    o.bucket_shift = int(bucket_shift)
    for k, v in (schedule or {}).items():  # coarse-peel schedule (see autotune.py)
        if k not in SCHEDULE_KEYS:
            raise ValueError(f"unknown schedule key {k}")
        setattr(o, k, int(v))
    o.recount = int(bool(recount))
    o.compact = int(bool(compact))
    o.mem = mem
    o.graph_rounds = int(bool(graph_rounds))
    if stream is not None:
        o.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    else:
        try:
            import torch
            o.stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            o.stream = None
    if bounds is not None:
        b = np.ascontiguousarray(bounds, dtype=np.uint64)
        if keep is not None:
            keep.append(b)
        o.bounds_mode = BOUNDS_EXPLICIT
        o.bounds = b.ctypes.data_as(ctypes.c_void_p)
        o.n_bounds = b.size
    if mlp is not None:  # (params tensor on the device, hidden, out)
        o.bounds_mode = BOUNDS_LEARNED
        o.learned_vet = float(learned_vet)
        o.mlp_params = ctypes.c_void_p(mlp[0].data_ptr())
        o.mlp_hidden, o.mlp_out = int(mlp[1]), int(mlp[2])
    if bounds_out is not None:
        o.bounds_out = bounds_out.ctypes.data_as(ctypes.c_void_p)
        o.n_bounds_out = bounds_out.size
    return o


def count(dg: DeviceGraph, vertices=True, edges=False, stream=None, with_stats=False, scratch=0):
    """Per-vertex (U and V) and per-edge butterfly counts (Alg. 1); scratch:
    the counters of the heavier starts (SCRATCH_*)."""
    import torch
    dev = dg.u_off.device
    cu = torch.empty(max(dg.nu, 1), dtype=torch.int64, device=dev) if vertices else None
    cv = torch.empty(max(dg.nv, 1), dtype=torch.int64, device=dev) if vertices else None
    ce = torch.empty(max(dg.m, 1), dtype=torch.int64, device=dev) if edges else None
    st = Stats()
    o = _opts(stream, schedule={"count_scratch": scratch})
    g = dg.c_struct()
    rc = lib().pbng_count(ctypes.byref(g), cu.data_ptr() if cu is not None else None,
                          cv.data_ptr() if cv is not None else None, ce.data_ptr() if ce is not None else None,
                          ctypes.byref(o), ctypes.byref(st))
    _check(rc, "pbng_count")
    out = (cu[:dg.nu] if cu is not None else None, cv[:dg.nv] if cv is not None else None,
           ce[:dg.m] if ce is not None else None)
    return (out, st.to_dict()) if with_stats else out


def _side(side) -> int:
    if side in ("U", "u", 0, SIDE_U):
        return SIDE_U
    if side in ("V", "v", 1, SIDE_V):
        return SIDE_V
    raise ValueError(side)


def tip_decompose(dg: DeviceGraph, side="U", P=150, bounds=None, recount=True, compact=True, graph_rounds=False,
                  stream=None, with_stats=False, mlp=None, bounds_out=None, bucket_shift=0, schedule=None,
                  learned_vet=0.0):
    """Tip numbers of one side (two-phase PBNG, Sec. 3.1-3.2).

    bounds: explicit upper bounds; mlp: (params, hidden, out) of the learned
    proposer, whose bounds the estimator judges (learned_vet: most work of a
    learned range as a multiple of the estimator's target, 0 = 2.0, negative
    = unjudged); bounds_out: numpy uint64 array receiving the bounds used."""
    import torch
    s = _side(side)
    n = dg.nu if s == SIDE_U else dg.nv
    out = torch.empty(max(n, 1), dtype=torch.int64, device=dg.u_off.device)
    keep = []
    o = _opts(stream, bounds, recount, compact, graph_rounds=graph_rounds, keep=keep, mlp=mlp, bounds_out=bounds_out,
              bucket_shift=bucket_shift, schedule=schedule, learned_vet=learned_vet)
    st = Stats()
    g = dg.c_struct()
    rc = lib().pbng_tip_decompose(ctypes.byref(g), s, int(P), out.data_ptr(), ctypes.byref(o), ctypes.byref(st))
    _check(rc, "pbng_tip_decompose")
    return (out[:n], st.to_dict()) if with_stats else out[:n]


def propose_bounds(dg: DeviceGraph, side="U", P=150, mlp=None, bounds=None, stream=None, **kw):
    """The P+1 coarse-phase bounds theta(1..P+1) (numpy uint64; unused ranges
    and theta(P+1) are 2^64-1) the estimator, or the learned proposer when
    ``mlp`` is given, would use (Sec. 3.1.3)."""
    out = np.zeros(int(P) + 1, dtype=np.uint64)
    keep = []
    o = _opts(stream, bounds, kw.get("recount", True), kw.get("compact", True), keep=keep, mlp=mlp,
              graph_rounds=kw.get("graph_rounds", False), schedule=kw.get("schedule"),
              learned_vet=kw.get("learned_vet", 0.0))
    g = dg.c_struct()
    _check(lib().pbng_propose_bounds(ctypes.byref(g), _side(side), int(P), out.ctypes.data, ctypes.byref(o)),
           "pbng_propose_bounds")
    return out


def be_index_sums(dg: DeviceGraph, stream=None, with_stats=False):
    """(per-edge sum over its blooms of k_B - 1, sum over blooms of C(k_B, 2)) of the BE-Index."""
    import torch
    out = torch.empty(max(dg.m, 1), dtype=torch.int64, device=dg.u_off.device)
    tot = ctypes.c_uint64(0)
    o = _opts(stream)
    st = Stats()
    g = dg.c_struct()
    _check(lib().pbng_be_index_sums(ctypes.byref(g), out.data_ptr(), ctypes.byref(tot), ctypes.byref(o),
                                    ctypes.byref(st)), "pbng_be_index_sums")
    res = (out[:dg.m], int(tot.value))
    return (res, st.to_dict()) if with_stats else res


def bound_features(dg: DeviceGraph, side="U", stream=None):
    """128 histogram features of the learned bound proposer (float32 tensor)."""
    import torch
    out = torch.zeros(128, dtype=torch.float32, device=dg.u_off.device)
    o = _opts(stream)
    g = dg.c_struct()
    _check(lib().pbng_bound_features(ctypes.byref(g), _side(side), out.data_ptr(), ctypes.byref(o)),
           "pbng_bound_features")
    return out


def wing_bound_features(dg: DeviceGraph, stream=None):
    """128 histogram features of the learned wing bound proposer (float32 tensor)."""
    import torch
    out = torch.zeros(128, dtype=torch.float32, device=dg.u_off.device)
    o = _opts(stream)
    g = dg.c_struct()
    _check(lib().pbng_wing_bound_features(ctypes.byref(g), out.data_ptr(), ctypes.byref(o)),
           "pbng_wing_bound_features")
    return out


def _cs(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def mlp_forward(params, dims, X, stream=None):
    """y = MLP(x) for the rows of X (device float32); dims = (in, hidden, out)."""
    import torch
    nin, hid, out = dims
    Y = torch.empty((X.shape[0], out), dtype=torch.float32, device=X.device)
    _check(lib().pbng_mlp_forward(params.data_ptr(), nin, hid, out, X.data_ptr(), X.shape[0], Y.data_ptr(), _cs(stream)),
           "pbng_mlp_forward")
    return Y


def mlp_grad(params, dims, X, T, stream=None):
    """(gradient of the mean squared error w.r.t. params, loss)."""
    import torch
    nin, hid, out = dims
    grad = torch.empty_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    _check(lib().pbng_mlp_grad(params.data_ptr(), nin, hid, out, X.data_ptr(), T.data_ptr(), X.shape[0],
                               grad.data_ptr(), loss.data_ptr(), _cs(stream)), "pbng_mlp_grad")
    return grad, float(loss.item())


def mlp_adam(params, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().pbng_mlp_adam(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(), params.numel(),
                               lr, beta1, beta2, eps, step, _cs(stream)), "pbng_mlp_adam")


def tip_decompose_host(g, side="U", P=150, with_stats=False, **kw):
    """Tip numbers with host input and output buffers (the library copies)."""
    s = _side(side)
    off = np.ascontiguousarray(g.u_off, dtype=np.uint64)
    adj = np.ascontiguousarray(g.u_adj, dtype=np.uint32)
    n = g.nu if s == SIDE_U else g.nv
    out = np.zeros(max(n, 1), dtype=np.uint64)
    o = _opts(kw.get("stream"), kw.get("bounds"), kw.get("recount", True), kw.get("compact", True), mem=MEM_HOST,
              graph_rounds=kw.get("graph_rounds", False), keep=[], bucket_shift=kw.get("bucket_shift", 0),
              schedule=kw.get("schedule"))
    st = Stats()
    cg = Bigraph(int(g.nu), int(g.nv), adj.size, off.ctypes.data, adj.ctypes.data if adj.size else 0)
    rc = lib().pbng_tip_decompose(ctypes.byref(cg), s, int(P), out.ctypes.data, ctypes.byref(o), ctypes.byref(st))
    _check(rc, "pbng_tip_decompose")
    return (out[:n], st.to_dict()) if with_stats else out[:n]


def wing_decompose(dg: DeviceGraph, P=400, bounds=None, recount=True, compact=True, stream=None, with_stats=False,
                   schedule=None, bounds_out=None, mlp=None, learned_vet=0.0):
    """Wing numbers of every edge (BE-Index PBNG, Sec. 3.3); mlp: (params,
    hidden, out) of the learned wing bound proposer, learned_vet as for
    tip_decompose."""
    import torch
    out = torch.empty(max(dg.m, 1), dtype=torch.int64, device=dg.u_off.device)
    keep = []
    o = _opts(stream, bounds, recount, compact, keep=keep, schedule=schedule, bounds_out=bounds_out, mlp=mlp,
              learned_vet=learned_vet)
    st = Stats()
    g = dg.c_struct()
    rc = lib().pbng_wing_decompose(ctypes.byref(g), int(P), out.data_ptr(), ctypes.byref(o), ctypes.byref(st))
    _check(rc, "pbng_wing_decompose")
    return (out[:dg.m], st.to_dict()) if with_stats else out[:dg.m]


def tip_decompose_batch(dgs, side="U", P=150, stream=None, with_stats=False, **kw):
    """Tip numbers of many independent graphs in one call (disjoint union)."""
    import torch
    s = _side(side)
    n = len(dgs)
    gs = (Bigraph * max(n, 1))(*[d.c_struct() for d in dgs])
    outs = [torch.empty(max(d.nu if s == SIDE_U else d.nv, 1), dtype=torch.int64, device=d.u_off.device) for d in dgs]
    ptrs = (ctypes.c_void_p * max(n, 1))(*[o.data_ptr() for o in outs])
    keep = []
    o = _opts(stream, kw.get("bounds"), kw.get("recount", True), kw.get("compact", True), keep=keep,
              graph_rounds=kw.get("graph_rounds", False), bucket_shift=kw.get("bucket_shift", 0),
              schedule=kw.get("schedule"), bounds_out=kw.get("bounds_out"))
    st = Stats()
    rc = lib().pbng_tip_decompose_batch(gs, n, s, int(P), ptrs, ctypes.byref(o), ctypes.byref(st))
    _check(rc, "pbng_tip_decompose_batch")
    res = [t[:(d.nu if s == SIDE_U else d.nv)] for t, d in zip(outs, dgs)]
    return (res, st.to_dict()) if with_stats else res


def wing_decompose_batch(dgs, P=400, stream=None, with_stats=False, **kw):
    """Wing numbers of many independent graphs in one call (disjoint union)."""
    import torch
    n = len(dgs)
    gs = (Bigraph * max(n, 1))(*[d.c_struct() for d in dgs])
    outs = [torch.empty(max(d.m, 1), dtype=torch.int64, device=d.u_off.device) for d in dgs]
    ptrs = (ctypes.c_void_p * max(n, 1))(*[o.data_ptr() for o in outs])
    o = _opts(stream, kw.get("bounds"), kw.get("recount", True), kw.get("compact", True), keep=[],
              bounds_out=kw.get("bounds_out"))
    st = Stats()
    rc = lib().pbng_wing_decompose_batch(gs, n, int(P), ptrs, ctypes.byref(o), ctypes.byref(st))
    _check(rc, "pbng_wing_decompose_batch")
    res = [t[:d.m] for t, d in zip(outs, dgs)]
    return (res, st.to_dict()) if with_stats else res


def _host_structs(graphs):
    keep, structs = [], []
    for g in graphs:
        off = np.ascontiguousarray(g.u_off, dtype=np.uint64)
        adj = np.ascontiguousarray(g.u_adj, dtype=np.uint32)
        keep += [off, adj]
        structs.append(Bigraph(int(g.nu), int(g.nv), adj.size, off.ctypes.data, adj.ctypes.data if adj.size else 0))
    return keep, (Bigraph * max(len(graphs), 1))(*structs)


def tip_decompose_batch_host(graphs, side="U", P=150, with_stats=False, **kw):
    """Batch tip numbers with host input and output buffers (the library copies)."""
    s = _side(side)
    keep, gs = _host_structs(graphs)
    outs = [np.zeros(max(g.nu if s == SIDE_U else g.nv, 1), dtype=np.uint64) for g in graphs]
    ptrs = (ctypes.c_void_p * max(len(graphs), 1))(*[o.ctypes.data for o in outs])
    o = _opts(kw.get("stream"), kw.get("bounds"), kw.get("recount", True), kw.get("compact", True), mem=MEM_HOST,
              keep=keep, graph_rounds=kw.get("graph_rounds", False), bounds_out=kw.get("bounds_out"))
    st = Stats()
    _check(lib().pbng_tip_decompose_batch(gs, len(graphs), s, int(P), ptrs, ctypes.byref(o), ctypes.byref(st)),
           "pbng_tip_decompose_batch")
    res = [t[:(g.nu if s == SIDE_U else g.nv)] for t, g in zip(outs, graphs)]
    return (res, st.to_dict()) if with_stats else res


def wing_decompose_batch_host(graphs, P=400, with_stats=False, **kw):
    """Batch wing numbers with host buffers; an edgeless graph gets a NULL output."""
    keep, gs = _host_structs(graphs)
    outs = [np.zeros(g.m, dtype=np.uint64) if g.m else None for g in graphs]
    ptrs = (ctypes.c_void_p * max(len(graphs), 1))(*[o.ctypes.data if o is not None else None for o in outs])
    o = _opts(kw.get("stream"), kw.get("bounds"), kw.get("recount", True), kw.get("compact", True), mem=MEM_HOST,
              keep=keep, bounds_out=kw.get("bounds_out"))
    st = Stats()
    _check(lib().pbng_wing_decompose_batch(gs, len(graphs), int(P), ptrs, ctypes.byref(o), ctypes.byref(st)),
           "pbng_wing_decompose_batch")
    res = [t if t is not None else np.zeros(0, dtype=np.uint64) for t in outs]
    return (res, st.to_dict()) if with_stats else res


def tip_components(dg: DeviceGraph, side, theta, k, stream=None, with_stats=False):
    """k-tips from tip numbers: per vertex of `side`, the smallest id of its
    k-tip (int32 tensor holding uint32; -1 = 0xffffffff for theta < k)."""
    import torch
    s = _side(side)
    n = dg.nu if s == SIDE_U else dg.nv
    th = theta.to(device=dg.u_off.device, dtype=torch.int64).contiguous()
    if th.numel() < n:
        raise ValueError("theta has fewer entries than the side has vertices")
    out = torch.empty(max(n, 1), dtype=torch.int32, device=dg.u_off.device)
    o = _opts(stream)
    st = Stats()
    g = dg.c_struct()
    rc = lib().pbng_tip_components(ctypes.byref(g), s, th.data_ptr(), int(k), out.data_ptr(), ctypes.byref(o),
                                   ctypes.byref(st))
    _check(rc, "pbng_tip_components")
    return (out[:n], st.to_dict()) if with_stats else out[:n]


def wing_components(dg: DeviceGraph, theta, k, stream=None, with_stats=False):
    """k-wings from wing numbers: per edge, the smallest edge id of its k-wing
    (int32 tensor holding uint32; -1 = 0xffffffff for theta < k)."""
    import torch
    th = theta.to(device=dg.u_off.device, dtype=torch.int64).contiguous()
    if th.numel() < dg.m:
        raise ValueError("theta has fewer entries than the graph has edges")
    out = torch.empty(max(dg.m, 1), dtype=torch.int32, device=dg.u_off.device)
    o = _opts(stream)
    st = Stats()
    g = dg.c_struct()
    rc = lib().pbng_wing_components(ctypes.byref(g), th.data_ptr(), int(k), out.data_ptr(), ctypes.byref(o),
                                    ctypes.byref(st))
    _check(rc, "pbng_wing_components")
    return (out[:dg.m], st.to_dict()) if with_stats else out[:dg.m]


def vertex_counts_noalloc(dg: DeviceGraph, dg_t: DeviceGraph, stream=None):
    """Per-vertex butterfly counts of dg's U side without any device
    allocation by the library (fixed static scratch; see include/pbng.h).
    ``dg_t`` is the transposed graph (its U-side CSR is dg's V-side CSR)."""
    import torch
    out = torch.empty(max(dg.nu, 1), dtype=torch.int64, device=dg.u_off.device)
    s = stream if stream is not None else torch.cuda.current_stream(dg.u_off.device)
    rc = lib().pbng_vertex_counts_noalloc(dg.nu, dg.nv, dg.m, dg.u_off.data_ptr(),
                                          dg.u_adj.data_ptr() if dg.m else None, dg_t.u_off.data_ptr(),
                                          dg_t.u_adj.data_ptr() if dg_t.m else None, out.data_ptr(),
                                          ctypes.c_void_p(s.cuda_stream))
    _check(rc, "pbng_vertex_counts_noalloc")
    return out[:dg.nu]
