"""Thin ctypes binding of libnk (include/nk.h): argument marshalling only.

Every computation runs in the CUDA library; there is no CPU fallback.  If
``_build/libnk.so`` is missing, importing the library raises (build it with
``python -m paper_1403_3005_gb300.build`` or ``__graft_entry__.build()``).

Host arrays are numpy arrays.  Device buffers may be passed as torch CUDA tensors
(their data pointers are handed to the library with the NK_RUN_DEVICE_PTRS flag);
PyTorch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libnk.so")

OK, PENDING = 0, 1
ERR_ARG, ERR_GRAPH, ERR_NOMEM, ERR_OVERFLOW, ERR_CUDA, ERR_TIMEOUT, ERR_SHUTDOWN = -1, -2, -3, -4, -5, -6, -7
CSR_VALIDATE, CSR_CANONICALISE, CSR_DEVICE_PTRS = 1, 2, 4
GEN_ER, GEN_BA, GEN_RMAT = 1, 2, 3
MODE_AUTO, MODE_PER_SOURCE, MODE_BATCHED = 0, 1, 2
DIR_AUTO, DIR_TOP_DOWN, DIR_BOTTOM_UP = 0, 1, 2
RUN_DEVICE_PTRS, RUN_TIME_KERNELS, RUN_CUDA_GRAPH, RUN_RELABEL, RUN_NO_RELABEL = 1, 2, 4, 8, 16

_NAMES = {OK: "NK_OK", PENDING: "NK_PENDING", ERR_ARG: "NK_ERR_ARG", ERR_GRAPH: "NK_ERR_GRAPH",
          ERR_NOMEM: "NK_ERR_NOMEM", ERR_OVERFLOW: "NK_ERR_OVERFLOW", ERR_CUDA: "NK_ERR_CUDA",
          ERR_TIMEOUT: "NK_ERR_TIMEOUT", ERR_SHUTDOWN: "NK_ERR_SHUTDOWN"}


class NkError(RuntimeError):
    def __init__(self, rc: int, msg: str):
        super().__init__(f"{_NAMES.get(rc, rc)}: {msg}")
        self.rc = rc


class RunOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("batch", ctypes.c_int32), ("tpv", ctypes.c_int32),
                ("direction", ctypes.c_int32), ("alpha", ctypes.c_double),
                ("flags", ctypes.c_uint32), ("grid_ctas", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


class RunStats(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("batch", ctypes.c_int32), ("tpv", ctypes.c_int32),
                ("max_depth", ctypes.c_int32), ("launches", ctypes.c_int64),
                ("kernel_ms", ctypes.c_double), ("td_levels", ctypes.c_int64),
                ("bu_levels", ctypes.c_int64), ("alpha", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_double), ("max_inflight", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("timeout_s", ctypes.c_double),
                ("no_pack", ctypes.c_int32), ("reserved", ctypes.c_int32 * 7)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("edges_x_sources", ctypes.c_double), ("peak_inflight", ctypes.c_int64),
                ("peak_bytes", ctypes.c_double), ("queue_p50_ms", ctypes.c_double),
                ("queue_p99_ms", ctypes.c_double), ("run_p50_ms", ctypes.c_double),
                ("run_p99_ms", ctypes.c_double), ("jobs", ctypes.c_int64),
                ("packed_requests", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# every function declared in include/nk.h: name -> (restype, argtypes)
_P, _I32, _I64, _U32, _U64, _D = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double)
_INT = ctypes.c_int
SIGNATURES = {
    "nk_graph_from_csr": (_INT, [_I32, _P, _P, _I64, _U32, _P]),
    "nk_graph_from_edges": (_INT, [_I32, _I64, _P, _P, _U32, _P]),
    "nk_graph_generate": (_INT, [_INT, _P, _I32, _U64, _P]),
    "nk_graph_info": (_INT, [_P, _P, _P]),
    "nk_graph_export_csr": (_INT, [_P, _P, _P]),
    "nk_graph_free": (_INT, [_P]),
    "nk_sample_sources": (_INT, [_I32, _U64, _I32, _P, _U32]),
    "nk_sssp": (_INT, [_P, _I32, _P, _P]),
    "nk_sssp_noalloc": (_INT, [_I32, _P, _P, _I64, _I32, _P, _P, _P]),
    "nk_betweenness_exact": (_INT, [_P, _P]),
    "nk_betweenness_sampled": (_INT, [_P, _U64, _I32, _P]),
    "nk_betweenness_sampled_opts": (_INT, [_P, _U64, _I32, _P, _P]),
    "nk_betweenness_sources": (_INT, [_P, _P, _I32, _D, _P, _P]),
    "nk_graph_set_weights": (_INT, [_P, _P, _U32]),
    "nk_graph_random_weights": (_INT, [_P, _U64, _I32]),
    "nk_graph_export_weights": (_INT, [_P, _P]),
    "nk_sssp_weighted": (_INT, [_P, _I32, _P, _P]),
    "nk_betweenness_weighted_exact": (_INT, [_P, _P]),
    "nk_betweenness_weighted_sampled": (_INT, [_P, _U64, _I32, _P, _P]),
    "nk_betweenness_rk": (_INT, [_P, ctypes.c_double, ctypes.c_double, _U64, _P, _P, _P, _P]),
    "nk_vertex_diameter_estimate": (_INT, [_P, _P]),
    "nk_edge_betweenness_exact": (_INT, [_P, _P]),
    "nk_edge_betweenness_sampled": (_INT, [_P, _U64, _I32, _P, _P]),
    "nk_closeness_exact": (_INT, [_P, _P, _P]),
    "nk_closeness_sampled": (_INT, [_P, _U64, _I32, _P, _P, _P]),
    "nk_last_run_stats": (_INT, [_P]),
    "nk_autotune": (_INT, [_P, _U64, _I32, _P]),
    "nk_server_create": (_INT, [_P, _P]),
    "nk_server_destroy": (None, [_P]),
    "nk_serve_submit": (_INT, [_P, _P, _U64, _I32, _P, _P]),
    "nk_serve_poll": (_INT, [_P, _I64]),
    "nk_serve_wait": (_INT, [_P, _I64, _D]),
    "nk_server_get_stats": (_INT, [_P, _P]),
    "nk_set_stream": (_INT, [_P]),
    "nk_set_wait_limit_ns": (_INT, [_U64]),
    "nk_selftest_wait_timeout": (_INT, [_U64]),
    "nk_launch_count": (_U64, []),
    "nk_alloc_count": (_U64, []),
    "nk_last_error": (ctypes.c_char_p, []),
    "nk_version": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def lib():
    """The loaded libnk.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libnk.so not built ({LIB_PATH} missing); run the package build")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype, f.argtypes = res, args
            _lib = L
        return _lib


def _check(rc: int) -> int:
    if rc < 0:
        raise NkError(rc, lib().nk_last_error().decode(errors="replace"))
    return rc


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _host_i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _dev_ptr(t):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device buffers must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- graphs
class Graph:
    """Owner of an nk_graph handle (a canonical CSR resident in GPU memory)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @property
    def handle(self):
        if not self._h:
            raise ValueError("graph was freed")
        return self._h

    def info(self):
        n, A = ctypes.c_int32(), ctypes.c_int64()
        _check(lib().nk_graph_info(self.handle, ctypes.byref(n), ctypes.byref(A)))
        return n.value, A.value

    @property
    def n(self) -> int:
        return self.info()[0]

    @property
    def n_arcs(self) -> int:
        return self.info()[1]

    def export_csr(self):
        n, A = self.info()
        rp = np.empty(n + 1, np.int32)
        col = np.empty(max(A, 1), np.int32)
        _check(lib().nk_graph_export_csr(self.handle, _np_ptr(rp), _np_ptr(col)))
        return rp, col[:A].copy()

    def free(self):
        if self._h:
            _check(lib().nk_graph_free(self._h))
            self._h = None

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.nk_graph_free(self._h)
        except Exception:
            pass


def _new_graph(fn, *args) -> Graph:
    h = ctypes.c_void_p()
    _check(fn(*args, ctypes.byref(h)))
    return Graph(h)


def graph_from_csr(row_ptr, col, flags: int = CSR_VALIDATE) -> Graph:
    if _is_torch(row_ptr):
        n, A = row_ptr.numel() - 1, col.numel()
        return _new_graph(lib().nk_graph_from_csr, n, _dev_ptr(row_ptr), _dev_ptr(col), A,
                          flags | CSR_DEVICE_PTRS)
    rp, c = _host_i32(row_ptr), _host_i32(col)
    return _new_graph(lib().nk_graph_from_csr, len(rp) - 1, _np_ptr(rp),
                      _np_ptr(c) if len(c) else None, len(c), flags)


def graph_from_edges(n: int, u, v) -> Graph:
    if _is_torch(u):
        return _new_graph(lib().nk_graph_from_edges, n, u.numel(), _dev_ptr(u), _dev_ptr(v),
                          CSR_DEVICE_PTRS)
    uu, vv = _host_i32(u), _host_i32(v)
    return _new_graph(lib().nk_graph_from_edges, n, len(uu), _np_ptr(uu) if len(uu) else None,
                      _np_ptr(vv) if len(vv) else None, 0)


def graph_generate(kind: str, size: int, seed: int, **p) -> Graph:
    """kind 'er' (size = n, avg_deg), 'ba' (size = n, m0) or 'rmat' (size = scale,
    edge_factor, a, b, c)."""
    if kind == "er":
        k, params = GEN_ER, [p.get("avg_deg", 8.0)]
    elif kind == "ba":
        k, params = GEN_BA, [float(p.get("m0", 8))]
    elif kind == "rmat":
        k, params = GEN_RMAT, [float(p.get("edge_factor", 16)), p.get("a", 0.57),
                               p.get("b", 0.19), p.get("c", 0.19)]
    else:
        raise ValueError(kind)
    arr = (ctypes.c_double * len(params))(*params)
    return _new_graph(lib().nk_graph_generate, k, arr, size, seed)


# ---------------------------------------------------------------- sampler / sssp
def sample_sources(n: int, seed: int, k: int, out=None):
    if out is not None and _is_torch(out):
        _check(lib().nk_sample_sources(n, seed, k, _dev_ptr(out), RUN_DEVICE_PTRS))
        return out
    src = np.empty(k, np.int32)
    _check(lib().nk_sample_sources(n, seed, k, _np_ptr(src), 0))
    return src


def sssp(g: Graph, s: int):
    """(dist int32[n], sigma uint64[n]) of the forward sweep from s."""
    n = g.n
    dist = np.empty(n, np.int32)
    sigma = np.empty(n, np.uint64)
    _check(lib().nk_sssp(g.handle, s, _np_ptr(dist), _np_ptr(sigma)))
    return dist, sigma


def _check_noalloc_buffers(row_ptr, col, dist, sigma):
    """Refuses buffers the allocation-free sweep would read or write out of bounds, before
    anything reaches the library: dtypes, sizes, contiguity, then that every tensor is a
    CUDA tensor on the current device."""
    import torch
    for name, t, dt in (("row_ptr", row_ptr, torch.int32), ("col", col, torch.int32),
                        ("dist", dist, torch.int32), ("sigma", sigma, torch.int64)):
        if not _is_torch(t):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt} (got {t.dtype})")
        if t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous 1-D tensor")
    n = row_ptr.numel() - 1
    if n < 1:
        raise ValueError("row_ptr needs n + 1 >= 2 entries")
    if dist.numel() != n or sigma.numel() != n:
        raise ValueError(f"dist and sigma need n = {n} entries (got {dist.numel()} and {sigma.numel()})")
    for name, t in (("row_ptr", row_ptr), ("col", col), ("dist", dist), ("sigma", sigma)):
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
    cur = torch.cuda.current_device()
    for name, t in (("row_ptr", row_ptr), ("col", col), ("dist", dist), ("sigma", sigma)):
        if t.device.index != cur:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")
    return n


def sssp_noalloc(row_ptr, col, s: int, dist, sigma, stream=None) -> None:
    """Allocation-free forward sweep into caller-owned CUDA tensors: row_ptr (int32,
    n+1) and col (int32) hold a canonical CSR on the device; dist (int32, n) and sigma
    (int64 storage read as uint64, n) receive the results.  See nk.h.  Buffers of the
    wrong type, size or device raise ValueError before any launch."""
    n = _check_noalloc_buffers(row_ptr, col, dist, sigma)
    h = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().nk_sssp_noalloc(n, _dev_ptr(row_ptr), _dev_ptr(col) if col.numel() else None,
                                 col.numel(), s, _dev_ptr(dist), _dev_ptr(sigma),
                                 ctypes.c_void_p(h)))


# ---------------------------------------------------------------- betweenness
def run_opts(mode=MODE_AUTO, batch=0, tpv=0, direction=DIR_AUTO, alpha=0.0, flags=0, grid_ctas=0,
             chunk=0) -> RunOpts:
    o = RunOpts()
    o.mode, o.batch, o.tpv, o.direction, o.alpha, o.flags = mode, batch, tpv, direction, alpha, flags
    o.grid_ctas, o.chunk = grid_ctas, chunk
    return o


def _out_scores(g: Graph, out, opts: RunOpts | None):
    """Output buffer: a CUDA tensor (device pointer), a float64 numpy array (host,
    e.g. a view of pinned memory) or None (a new host array)."""
    if out is not None and _is_torch(out):
        o = run_opts() if opts is None else RunOpts.from_buffer_copy(opts)
        o.flags |= RUN_DEVICE_PTRS
        return _dev_ptr(out), o, out
    if opts is not None and (opts.flags & RUN_DEVICE_PTRS):
        opts = RunOpts.from_buffer_copy(opts)
        opts.flags &= ~RUN_DEVICE_PTRS
    if out is not None:
        if out.dtype != np.float64 or not out.flags.c_contiguous or len(out) != g.n:
            raise ValueError("host output must be a contiguous float64 array of n entries")
        return _np_ptr(out), opts, out
    arr = np.empty(g.n, np.float64)
    return _np_ptr(arr), opts, arr


def betweenness_exact(g: Graph) -> np.ndarray:
    out = np.empty(g.n, np.float64)
    _check(lib().nk_betweenness_exact(g.handle, _np_ptr(out)))
    return out


def betweenness_sampled(g: Graph, seed: int, k: int, opts: RunOpts | None = None, out=None):
    ptr, o, res = _out_scores(g, out, opts)
    _check(lib().nk_betweenness_sampled_opts(g.handle, seed, k, ptr,
                                              ctypes.byref(o) if o is not None else None))
    return res


def betweenness_sources(g: Graph, src, scale: float, opts: RunOpts | None = None, out=None):
    ptr, o, res = _out_scores(g, out, opts)
    if _is_torch(src):
        if o is None or not (o.flags & RUN_DEVICE_PTRS):
            raise ValueError("device sources need a device output tensor")
        sp, k = _dev_ptr(src), src.numel()
    else:
        s = _host_i32(src)
        if o is not None and (o.flags & RUN_DEVICE_PTRS):
            raise ValueError("host sources need a host output")
        sp, k = _np_ptr(s), len(s)
        src = s
    _check(lib().nk_betweenness_sources(g.handle, sp, k, scale, ptr,
                                         ctypes.byref(o) if o is not None else None))
    return res


# ---------------------------------------------------------------- several GPUs (Section 3.2)
def source_shard(src, rank: int, world: int):
    """Contiguous slice `rank` of `world` of one source set: entries [k r / N, k (r+1) / N).
    Sources are independent (Section 3.2), so the slices' dependency sums add up to the
    whole set's."""
    k = len(src)
    return src[k * rank // world:k * (rank + 1) // world]


def sharded_betweenness(n: int, src, rank: int, world: int, compute, group=None):
    """One sampled estimate split over the ranks of a torch.distributed group: rank r
    computes the unscaled dependency sums of its slice of the source set `src`
    (compute(slice) -> float64 tensor of n entries, or None for an empty slice), one sum
    all-reduce of the n-vector combines the ranks (the paper's per-thread arrays summed,
    Section 3.2), and the sum is scaled by n / (2k).  Every rank returns the estimate."""
    import torch
    import torch.distributed as dist
    part = source_shard(src, rank, world)
    local = compute(part) if len(part) else None
    if local is None:
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
        local = torch.zeros(n, dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(local, op=dist.ReduceOp.SUM, group=group)
    local.mul_(n / (2.0 * len(src)))
    return local


def betweenness_sampled_sharded(g: Graph, seed: int, k: int, opts: RunOpts | None = None, group=None,
                                out=None):
    """nk_betweenness_sampled split over the GPUs of a torch.distributed (NCCL) group,
    one GPU per rank, each holding its own copy of the graph: the k sources of
    nk_sample_sources(n, seed, k) are sampled on every rank, rank r sweeps its contiguous
    slice with nk_betweenness_sources (scale 1) into a device vector, one NCCL all-reduce
    sums the n-vectors, and the sum is scaled by n / (2k).  Returns the estimate (a CUDA
    tensor of n doubles) on every rank."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    n = g.n
    dev = torch.device("cuda", torch.cuda.current_device())
    src = sample_sources(n, seed, k, out=torch.empty(k, dtype=torch.int32, device=dev))
    res = out if out is not None else torch.empty(n, dtype=torch.float64, device=dev)

    def compute(part):
        betweenness_sources(g, part, 1.0, opts, out=res)
        return res
    return sharded_betweenness(n, src, rank, world, compute, group)


def set_weights(g: Graph, w) -> None:
    """Arc weights (int32 >= 1, equal on both arcs of an edge): numpy array or CUDA tensor."""
    if _is_torch(w):
        _check(lib().nk_graph_set_weights(g.handle, _dev_ptr(w), CSR_DEVICE_PTRS))
    else:
        wh = _host_i32(w)
        _check(lib().nk_graph_set_weights(g.handle, _np_ptr(wh), 0))


def random_weights(g: Graph, seed: int, wmax: int) -> None:
    _check(lib().nk_graph_random_weights(g.handle, seed, wmax))


def export_weights(g: Graph) -> np.ndarray:
    A = _arc_count(g)
    w = np.empty(max(A, 1), np.int32)
    _check(lib().nk_graph_export_weights(g.handle, _np_ptr(w)))
    return w[:A]


def sssp_weighted(g: Graph, s: int):
    dist = np.empty(g.n, np.int64)
    sigma = np.empty(g.n, np.uint64)
    _check(lib().nk_sssp_weighted(g.handle, s, _np_ptr(dist), _np_ptr(sigma)))
    return dist, sigma


def betweenness_weighted_exact(g: Graph) -> np.ndarray:
    out = np.empty(g.n, np.float64)
    _check(lib().nk_betweenness_weighted_exact(g.handle, _np_ptr(out)))
    return out


def betweenness_weighted_sampled(g: Graph, seed: int, k: int, opts: RunOpts | None = None, out=None):
    ptr, o, res = _out_scores(g, out, opts)
    _check(lib().nk_betweenness_weighted_sampled(g.handle, seed, k, ptr,
                                                 ctypes.byref(o) if o is not None else None))
    return res


def vertex_diameter_estimate(g: Graph) -> int:
    vd = ctypes.c_int32()
    _check(lib().nk_vertex_diameter_estimate(g.handle, ctypes.byref(vd)))
    return vd.value


def betweenness_rk(g: Graph, epsilon: float, delta: float, seed: int, opts: RunOpts | None = None,
                   out=None):
    """(scores, r, vd): the error-bounded estimate after Riondato and Kornaropoulos, on the
    scale of the exact unordered scores."""
    ptr, o, res = _out_scores(g, out, opts)
    r, vd = ctypes.c_int64(), ctypes.c_int32()
    _check(lib().nk_betweenness_rk(g.handle, epsilon, delta, seed, ptr, ctypes.byref(r), ctypes.byref(vd),
                                   ctypes.byref(o) if o is not None else None))
    return res, r.value, vd.value


def _arc_count(g: Graph) -> int:
    return g.info()[1]


def edge_betweenness_exact(g: Graph) -> np.ndarray:
    """Edge betweenness per arc of the canonical CSR (both arcs of an edge equal)."""
    out = np.empty(max(_arc_count(g), 1), np.float64)
    _check(lib().nk_edge_betweenness_exact(g.handle, _np_ptr(out)))
    return out[:_arc_count(g)]


def edge_betweenness_sampled(g: Graph, seed: int, k: int, opts: RunOpts | None = None, out=None):
    """Sampled edge betweenness per arc (scale n/(2k)); out: None (new host array) or a
    float64 CUDA tensor of A entries."""
    A = _arc_count(g)
    if out is not None:
        if not _is_torch(out) or out.numel() != A:
            raise ValueError("out must be a CUDA tensor of A entries")
        o = run_opts() if opts is None else RunOpts.from_buffer_copy(opts)
        o.flags |= RUN_DEVICE_PTRS
        _check(lib().nk_edge_betweenness_sampled(g.handle, seed, k, _dev_ptr(out), ctypes.byref(o)))
        return out
    res = np.empty(max(A, 1), np.float64)
    if opts is not None and (opts.flags & RUN_DEVICE_PTRS):
        opts = RunOpts.from_buffer_copy(opts)
        opts.flags &= ~RUN_DEVICE_PTRS
    _check(lib().nk_edge_betweenness_sampled(g.handle, seed, k, _np_ptr(res),
                                             ctypes.byref(opts) if opts is not None else None))
    return res[:A]


def closeness_exact(g: Graph):
    """(far, reach) over all sources: sum of distances and count of sources reaching
    each vertex; closeness = reach / far."""
    far = np.empty(g.n, np.float64)
    reach = np.empty(g.n, np.float64)
    _check(lib().nk_closeness_exact(g.handle, _np_ptr(far), _np_ptr(reach)))
    return far, reach


def closeness_sampled(g: Graph, seed: int, k: int, opts: RunOpts | None = None, out=None):
    """(far, reach) from k sampled sources, scaled by n/k (Eppstein-Wang estimate).
    out: None (new host arrays) or a pair of float64 CUDA tensors of n entries."""
    if out is not None:
        far, reach = out
        if not (_is_torch(far) and _is_torch(reach)):
            raise ValueError("out must be a pair of CUDA tensors")
        o = run_opts() if opts is None else RunOpts.from_buffer_copy(opts)
        o.flags |= RUN_DEVICE_PTRS
        _check(lib().nk_closeness_sampled(g.handle, seed, k, _dev_ptr(far), _dev_ptr(reach),
                                          ctypes.byref(o)))
        return far, reach
    far = np.empty(g.n, np.float64)
    reach = np.empty(g.n, np.float64)
    if opts is not None and (opts.flags & RUN_DEVICE_PTRS):
        opts = RunOpts.from_buffer_copy(opts)
        opts.flags &= ~RUN_DEVICE_PTRS
    _check(lib().nk_closeness_sampled(g.handle, seed, k, _np_ptr(far), _np_ptr(reach),
                                      ctypes.byref(opts) if opts is not None else None))
    return far, reach


def last_run_stats() -> dict:
    st = RunStats()
    _check(lib().nk_last_run_stats(ctypes.byref(st)))
    return st.as_dict()


def autotune(g: Graph, seed: int, k: int) -> RunOpts:
    o = RunOpts()
    _check(lib().nk_autotune(g.handle, seed, k, ctypes.byref(o)))
    return o


# ---------------------------------------------------------------- serving
class Server:
    """Continuous-batching betweenness server (nk_server_*)."""

    def __init__(self, mem_budget_bytes=0.0, max_inflight=0, batch=0, timeout_s=0.0, pack=True):
        o = ServerOpts()
        o.mem_budget_bytes, o.max_inflight, o.batch, o.timeout_s = (
            mem_budget_bytes, max_inflight, batch, timeout_s)
        o.no_pack = 0 if pack else 1
        h = ctypes.c_void_p()
        _check(lib().nk_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._bufs = {}

    def submit(self, g: Graph, seed: int, k: int):
        """Queues a sampled-betweenness request; returns (id, scores array)."""
        out = np.zeros(g.n, np.float64)
        rid = ctypes.c_int64()
        _check(lib().nk_serve_submit(self._h, g.handle, seed, k, _np_ptr(out), ctypes.byref(rid)))
        self._bufs[rid.value] = (out, g)
        return rid.value, out

    def poll(self, rid: int) -> int:
        rc = lib().nk_serve_poll(self._h, rid)
        if rc != PENDING:
            self._bufs.pop(rid, None)
        return rc

    def wait(self, rid: int, timeout_s: float = 60.0) -> int:
        rc = lib().nk_serve_wait(self._h, rid, timeout_s)
        if rc != PENDING:
            self._bufs.pop(rid, None)
        return rc

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().nk_server_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self._h:
            lib().nk_server_destroy(self._h)
            self._h = None
            self._bufs.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- misc
def set_stream(stream) -> None:
    """Orders every later call on a torch.cuda.Stream (or a raw cudaStream_t int)."""
    h = stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else 0)
    _check(lib().nk_set_stream(ctypes.c_void_p(h)))


def set_wait_limit_ns(ns: int) -> None:
    _check(lib().nk_set_wait_limit_ns(ns))


def selftest_wait_timeout(limit_ns: int) -> int:
    return lib().nk_selftest_wait_timeout(limit_ns)


def alloc_count() -> int:
    """Memory allocation calls the library has made in this process."""
    return int(lib().nk_alloc_count())


def launch_count() -> int:
    return int(lib().nk_launch_count())


def last_error() -> str:
    return lib().nk_last_error().decode(errors="replace")


def version() -> str:
    return lib().nk_version().decode()
