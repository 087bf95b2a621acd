"""ctypes front end of the sequential CPU oracle (``oracle/nk_oracle.c``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the cpu_baseline /
reference leg of ``bench.py`` are the only callers.  The product library never imports
this package, and this package never imports the product library.

Every function mirrors one C function and cites the passage of the paper it follows:
Brandes' algorithm, the sampled estimate and the error-bounded estimate after Riondato
and Kornaropoulos (Section 3.2, Table 1), BFS for unweighted
graphs and Dijkstra for weighted ones (Section 3.4), edge betweenness (Section 4.3), closeness exact and sampled (Table 1),
the generators of Section 5 (Table 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nk_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_GRAPH, ERR_NOMEM, ERR_OVERFLOW = 0, -1, -2, -3, -4


class OracleError(RuntimeError):
    def __init__(self, rc: int, what: str):
        super().__init__(f"oracle {what} failed with code {rc}")
        self.rc = rc


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (contraction off: the ER skip arithmetic is then the
    same sequence of IEEE operations on x86 and Arm hosts)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _bind(lib):
    """Declares the C signatures on a loaded copy of the oracle library."""
    i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    P = ctypes.c_void_p
    sig = {
        "or_mix64": (u64, [u64]),
        "or_stream": (u64, [u64, u64]),
        "or_log": (dbl, [dbl]),
        "or_gen_er": (i64, [i32, dbl, u64, P, P, i64]),
        "or_gen_ba": (i64, [i32, i32, u64, P, P, i64]),
        "or_gen_rmat": (i64, [i32, i32, dbl, dbl, dbl, u64, P, P, i64]),
        "or_csr_build": (i64, [i32, i64, P, P, P, P]),
        "or_sample_sources": (ctypes.c_int, [i32, u64, i32, P]),
        "or_bfs": (ctypes.c_int, [i32, P, P, i32, P, P]),
        "or_dependencies": (ctypes.c_int, [i32, P, P, i32, P]),
        "or_betweenness": (ctypes.c_int, [i32, P, P, i32, P, dbl, P]),
        "or_betweenness_exact": (ctypes.c_int, [i32, P, P, P]),
        "or_betweenness_sampled": (ctypes.c_int, [i32, P, P, u64, i32, P]),
        "or_closeness": (ctypes.c_int, [i32, P, P, i32, P, dbl, P, P]),
        "or_edge_betweenness": (ctypes.c_int, [i32, P, P, i32, P, dbl, P]),
        "or_vertex_diameter_estimate": (ctypes.c_int, [i32, P, P, P]),
        "or_edge_weights": (ctypes.c_int, [i32, P, P, u64, i32, P]),
        "or_sssp_weighted": (ctypes.c_int, [i32, P, P, P, i32, P, P]),
        "or_betweenness_weighted": (ctypes.c_int, [i32, P, P, P, i32, P, dbl, P]),
        "or_rk_sample_count": (i64, [dbl, dbl, i32]),
        "or_rk_path": (i32, [i32, P, P, u64, i64, P, P]),
        "or_rk_counts": (ctypes.c_int, [i32, P, P, u64, i64, i64, P]),
        "or_betweenness_rk": (ctypes.c_int, [i32, P, P, dbl, dbl, u64, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------- random numbers
def mix64(z: int) -> int:
    return int(_load().or_mix64(z))


def stream(seed: int, i: int) -> int:
    """i-th output of SplitMix64 seeded with ``seed`` (Steele, Lea, Flood 2014)."""
    return int(_load().or_stream(seed, i))


def log(x: float) -> float:
    """The ER generator's logarithm (atanh series), for 0 < x <= 1."""
    return float(_load().or_log(x))


# ---------------------------------------------------------------- generators (Section 5)
def _two_pass(fn, *args):
    m = fn(*args, None, None, 0)
    if m < 0:
        raise OracleError(m, fn.__name__)
    eu = np.empty(max(m, 1), np.int32)
    ev = np.empty(max(m, 1), np.int32)
    m2 = fn(*args, _p(eu), _p(ev), m)
    assert m2 == m
    return eu[:m], ev[:m]


def gen_er(n: int, avg_deg: float, seed: int):
    """Erdos-Renyi G(n, p = avg_deg/(n-1)) by chunked geometric skipping."""
    return _two_pass(_load().or_gen_er, n, avg_deg, seed)


def gen_ba(n: int, m0: int, seed: int):
    """Barabasi-Albert linear preferential attachment, m0 edges per new vertex."""
    return _two_pass(_load().or_gen_ba, n, m0, seed)


def gen_rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int):
    """R-MAT with 2^scale vertices and edge_factor * 2^scale raw edges."""
    return _two_pass(_load().or_gen_rmat, scale, edge_factor, a, b, c, seed)


def csr_build(n: int, eu, ev):
    """Canonical CSR (symmetrised, no self-loops, sorted, no duplicates)."""
    eu, ev = _i32(eu), _i32(ev)
    m = len(eu)
    rp = np.empty(n + 1, np.int32)
    col = np.empty(max(2 * m, 1), np.int32)
    A = _load().or_csr_build(n, m, _p(eu), _p(ev), _p(rp), _p(col))
    if A < 0:
        raise OracleError(A, "csr_build")
    return rp, col[:A].copy()


def generate(kind: str, size: int, seed: int, **params):
    """Raw edges of one of the three generators, then the canonical CSR: (n, rp, col)."""
    if kind == "er":
        eu, ev = gen_er(size, params.get("avg_deg", 8.0), seed)
        n = size
    elif kind == "ba":
        eu, ev = gen_ba(size, int(params.get("m0", 8)), seed)
        n = size
    elif kind == "rmat":
        eu, ev = gen_rmat(size, int(params.get("edge_factor", 16)), params.get("a", 0.57),
                          params.get("b", 0.19), params.get("c", 0.19), seed)
        n = 1 << size
    else:
        raise ValueError(kind)
    rp, col = csr_build(n, eu, ev)
    return n, rp, col


# ---------------------------------------------------------------- sampler (Section 3.2)
def sample_sources(n: int, seed: int, k: int) -> np.ndarray:
    src = np.empty(k, np.int32)
    rc = _load().or_sample_sources(n, seed, k, _p(src))
    if rc:
        raise OracleError(rc, "sample_sources")
    return src


# ---------------------------------------------------------------- BFS / Brandes
def bfs(rp, col, s: int):
    """(dist int32[n], sigma uint64[n]) from source s; raises on sigma overflow."""
    rp, col = _i32(rp), _i32(col)
    n = len(rp) - 1
    dist = np.empty(n, np.int32)
    sigma = np.empty(n, np.uint64)
    rc = _load().or_bfs(n, _p(rp), _p(col), s, _p(dist), _p(sigma))
    if rc:
        raise OracleError(rc, "bfs")
    return dist, sigma


def dependencies(rp, col, s: int) -> np.ndarray:
    rp, col = _i32(rp), _i32(col)
    n = len(rp) - 1
    delta = np.empty(n, np.float64)
    rc = _load().or_dependencies(n, _p(rp), _p(col), s, _p(delta))
    if rc:
        raise OracleError(rc, "dependencies")
    return delta


def betweenness_sources(rp, col, src, scale: float) -> np.ndarray:
    rp, col, src = _i32(rp), _i32(col), _i32(src)
    n = len(rp) - 1
    out = np.empty(n, np.float64)
    rc = _load().or_betweenness(n, _p(rp), _p(col), len(src), _p(src), scale, _p(out))
    if rc:
        raise OracleError(rc, "betweenness")
    return out


def betweenness_exact(rp, col) -> np.ndarray:
    rp, col = _i32(rp), _i32(col)
    n = len(rp) - 1
    out = np.empty(n, np.float64)
    rc = _load().or_betweenness_exact(n, _p(rp), _p(col), _p(out))
    if rc:
        raise OracleError(rc, "betweenness_exact")
    return out


def betweenness_sampled(rp, col, seed: int, k: int) -> np.ndarray:
    rp, col = _i32(rp), _i32(col)
    n = len(rp) - 1
    out = np.empty(n, np.float64)
    rc = _load().or_betweenness_sampled(n, _p(rp), _p(col), seed, k, _p(out))
    if rc:
        raise OracleError(rc, "betweenness_sampled")
    return out


# ---------------------------------------------------------------- edge betweenness (Section 4.3)
def edge_betweenness_sources(rp, col, src, scale: float) -> np.ndarray:
    """Per arc j of the CSR: scale * (sum over the arc + sum over its reverse arc) of the
    shares sigma_v / sigma_w * (1 + delta_w); both arcs of an edge hold the edge's score."""
    rp, col, src = _i32(rp), _i32(col), _i32(src)
    n = len(rp) - 1
    out = np.empty(max(len(col), 1), np.float64)
    rc = _load().or_edge_betweenness(n, _p(rp), _p(col), len(src), _p(src), scale, _p(out))
    if rc:
        raise OracleError(rc, "edge_betweenness")
    return out[:len(col)]


def edge_betweenness_exact(rp, col) -> np.ndarray:
    n = len(rp) - 1
    return edge_betweenness_sources(rp, col, np.arange(n, dtype=np.int32), 0.5)


def edge_betweenness_sampled(rp, col, seed: int, k: int) -> np.ndarray:
    n = len(rp) - 1
    return edge_betweenness_sources(rp, col, sample_sources(n, seed, k), n / (2.0 * k))


# ---------------------------------------------------------------- error-bounded estimate (Section 3.2)
def vertex_diameter_estimate(rp, col) -> int:
    """Upper bound on the vertices of a shortest path: per component, min(|C|, 2 ecc(x) + 1)
    with x its smallest vertex; the largest over the components."""
    rp, col = _i32(rp), _i32(col)
    vd = ctypes.c_int32()
    rc = _load().or_vertex_diameter_estimate(len(rp) - 1, _p(rp), _p(col), ctypes.byref(vd))
    if rc:
        raise OracleError(rc, "vertex_diameter_estimate")
    return vd.value


def rk_sample_count(eps: float, delta: float, vd: int) -> int:
    r = _load().or_rk_sample_count(eps, delta, vd)
    if r < 0:
        raise OracleError(r, "rk_sample_count")
    return int(r)


def rk_path(rp, col, seed: int, i: int):
    """(u, v, interior) of sample i: the ordered pair and the interior vertices of its path
    from v towards u (None if v is not reachable from u)."""
    rp, col = _i32(rp), _i32(col)
    n = len(rp) - 1
    path = np.empty(n, np.int32)
    uv = np.empty(2, np.int32)
    L = _load().or_rk_path(n, _p(rp), _p(col), seed, i, _p(uv), _p(path))
    if L < -1:
        raise OracleError(L, "rk_path")
    return int(uv[0]), int(uv[1]), (None if L == -1 else path[:L].copy())


def rk_counts(rp, col, seed: int, i0: int, i1: int) -> np.ndarray:
    """Interior-vertex counts of samples i0 <= i < i1 (uint64[n])."""
    rp, col = _i32(rp), _i32(col)
    n = len(rp) - 1
    out = np.zeros(n, np.uint64)
    rc = _load().or_rk_counts(n, _p(rp), _p(col), seed, i0, i1, _p(out))
    if rc:
        raise OracleError(rc, "rk_counts")
    return out


def betweenness_rk(rp, col, eps: float, delta: float, seed: int):
    """(scores, r, vd): the Riondato-Kornaropoulos estimate on the scale of the exact
    unordered scores."""
    rp, col = _i32(rp), _i32(col)
    n = len(rp) - 1
    out = np.empty(n, np.float64)
    r, vd = ctypes.c_int64(), ctypes.c_int32()
    rc = _load().or_betweenness_rk(n, _p(rp), _p(col), eps, delta, seed, _p(out),
                                   ctypes.byref(r), ctypes.byref(vd))
    if rc:
        raise OracleError(rc, "betweenness_rk")
    return out, r.value, vd.value


# ---------------------------------------------------------------- weighted graphs (Sections 2.3, 3.4)
def edge_weights(rp, col, seed: int, wmax: int) -> np.ndarray:
    """Per arc: the edge {u, v} (u < v) weighs 1 + below(stream(seed, u 2^32 + v), wmax)."""
    rp, col = _i32(rp), _i32(col)
    w = np.empty(max(len(col), 1), np.int32)
    rc = _load().or_edge_weights(len(rp) - 1, _p(rp), _p(col), seed, wmax, _p(w))
    if rc:
        raise OracleError(rc, "edge_weights")
    return w[:len(col)]


def sssp_weighted(rp, col, w, s: int):
    """(dist int64[n] (-1 unreachable), sigma uint64[n]) by Dijkstra from s."""
    rp, col, w = _i32(rp), _i32(col), _i32(w)
    n = len(rp) - 1
    dist = np.empty(n, np.int64)
    sigma = np.empty(n, np.uint64)
    rc = _load().or_sssp_weighted(n, _p(rp), _p(col), _p(w), s, _p(dist), _p(sigma))
    if rc:
        raise OracleError(rc, "sssp_weighted")
    return dist, sigma


def betweenness_weighted_sources(rp, col, w, src, scale: float) -> np.ndarray:
    rp, col, w, src = _i32(rp), _i32(col), _i32(w), _i32(src)
    n = len(rp) - 1
    out = np.empty(n, np.float64)
    rc = _load().or_betweenness_weighted(n, _p(rp), _p(col), _p(w), len(src), _p(src), scale, _p(out))
    if rc:
        raise OracleError(rc, "betweenness_weighted")
    return out


def betweenness_weighted_exact(rp, col, w) -> np.ndarray:
    n = len(rp) - 1
    return betweenness_weighted_sources(rp, col, w, np.arange(n, dtype=np.int32), 0.5)


def betweenness_weighted_sampled(rp, col, w, seed: int, k: int) -> np.ndarray:
    n = len(rp) - 1
    return betweenness_weighted_sources(rp, col, w, sample_sources(n, seed, k), n / (2.0 * k))


# ---------------------------------------------------------------- closeness (Table 1)
def closeness_sources(rp, col, src, scale: float):
    """(far, reach): scale * sum of d(s, v), and scale * count, over sources s != v
    that reach v."""
    rp, col, src = _i32(rp), _i32(col), _i32(src)
    n = len(rp) - 1
    far = np.empty(n, np.float64)
    reach = np.empty(n, np.float64)
    rc = _load().or_closeness(n, _p(rp), _p(col), len(src), _p(src), scale, _p(far), _p(reach))
    if rc:
        raise OracleError(rc, "closeness")
    return far, reach


def closeness_exact(rp, col):
    n = len(rp) - 1
    return closeness_sources(rp, col, np.arange(n, dtype=np.int32), 1.0)


def closeness_sampled(rp, col, seed: int, k: int):
    n = len(rp) - 1
    return closeness_sources(rp, col, sample_sources(n, seed, k), n / k)
