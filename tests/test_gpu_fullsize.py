"""Parity at the benchmark workloads' full sizes, in the launch configuration bench.py
times (batched form, autotuned batch and switch threshold).

Where the oracle can compute outputs one by one (a source subset of the same sampled
set, on the oracle's own copy of the graph), they are compared element by element;
otherwise properties that hold at any size are checked on the GPU outputs.  The oracle
never receives a GPU output.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
RTOL, ATOL = 1e-9, 1e-12


@pytest.fixture(scope="module")
def nk():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    from paper_1403_3005_gb300 import nk as _nk
    _nk.lib()
    return _nk


def close(a, b):
    return np.allclose(a, b, rtol=RTOL, atol=ATOL)


def _slices(fn, items, threads=None):
    """The oracle on slices of `items` in host threads (the calls release the GIL)."""
    import concurrent.futures as cf
    import os
    t = threads or max(2, min(16, os.cpu_count() or 2))
    parts = [p for p in np.array_split(items, t) if len(p)]
    with cf.ThreadPoolExecutor(len(parts)) as ex:
        return list(ex.map(fn, parts))


def test_rmat18_sampled_k1024_full_vector(nk):
    # the default bench workload: every score of the k = 1024 sampled estimate
    g = nk.graph_generate("rmat", 18, 1)
    n, rp, col = oracle.generate("rmat", 18, 1)
    opts = nk.autotune(g, 2, 1024)
    got = nk.betweenness_sampled(g, 2, 1024, opts)
    src = oracle.sample_sources(n, 2, 1024)
    # the oracle on 4 slices of the source set, summed (sources are independent)
    import concurrent.futures as cf
    parts = np.array_split(src, 4)
    with cf.ThreadPoolExecutor(4) as ex:
        sums = list(ex.map(lambda p: oracle.betweenness_sources(rp, col, p, 1.0), parts))
    want = sum(sums) * (n / (2.0 * 1024))
    assert close(got, want)


def test_ba_1m_sources_subset(nk):
    # BA n = 1e6, m0 = 8: 96 sources of the k = 4096 sample (one full batch + a ragged one)
    # at default options, and in the autotuned setting that bench.py --config ba1m times
    g = nk.graph_generate("ba", 1000000, 1, m0=8)
    n, rp, col = oracle.generate("ba", 1000000, 1, m0=8)
    src = oracle.sample_sources(n, 2, 4096)[:96]
    want = sum(_slices(lambda p: oracle.betweenness_sources(rp, col, p, 1.0), src, threads=8))
    for batch in (64, 128):
        got = nk.betweenness_sources(g, src, 1.0, nk.run_opts(mode=nk.MODE_BATCHED, batch=batch))
        assert close(got, want), batch
    tuned = nk.autotune(g, 2, 4096)
    assert close(nk.betweenness_sources(g, src, 1.0, tuned), want), (tuned.batch, tuned.alpha, tuned.chunk)
    got = nk.betweenness_sources(g, src[:8], 1.0, nk.run_opts(mode=nk.MODE_PER_SOURCE))
    assert close(got, oracle.betweenness_sources(rp, col, src[:8], 1.0))
    g.free()


def test_rmat24_first_16_sources_autotuned(nk):
    # R-MAT scale 24, the headline workload: the scores of the first 16 sources of the
    # k = 8192 sample, element by element against the oracle on its own copy of the graph, in
    # the autotuned setting that bench.py times (n * B reaches 2^31 here: 2^24 x 128)
    g = nk.graph_generate("rmat", 24, 1)
    tuned = nk.autotune(g, 2, 8192)
    n, rp, col = oracle.generate("rmat", 24, 1)
    src = oracle.sample_sources(n, 2, 8192)[:16]
    got = nk.betweenness_sources(g, src, 1.0, tuned)
    g.free()
    want = sum(_slices(lambda p: oracle.betweenness_sources(rp, col, p, 1.0), src, threads=8))
    assert close(got, want), (tuned.batch, tuned.alpha, tuned.chunk, tuned.flags)


def test_rmat24_csr_properties(nk):
    # R-MAT scale 24: the raw edges the oracle computes one by one are in the GPU CSR, and the
    # CSR is canonical
    g = nk.graph_generate("rmat", 24, 1)
    n, A = g.info()
    rp, col = g.export_csr()
    g.free()
    assert rp[0] == 0 and rp[-1] == A and A % 2 == 0
    deg = np.diff(rp).astype(np.int64)
    # sample rows: sorted, no duplicates, no self-loop, symmetric
    rng = np.random.default_rng(0)
    for v in rng.choice(np.flatnonzero(deg > 0), 2000, replace=False):
        row = col[rp[v]:rp[v + 1]]
        assert np.all(np.diff(row) > 0) and not np.any(row == v)
        for w in row[:4]:
            r2 = col[rp[w]:rp[w + 1]]
            assert r2[np.searchsorted(r2, v)] == v
    # the first 20000 raw edges, computed by the oracle, are present
    from oracle import _load
    import ctypes
    E = 20000
    u = np.empty(E, np.int32)
    w = np.empty(E, np.int32)
    L = _load()
    L.or_gen_rmat(24, 16, 0.57, 0.19, 0.19, 1, u.ctypes.data_as(ctypes.c_void_p),
                  w.ctypes.data_as(ctypes.c_void_p), E)
    for a, b in zip(u.tolist(), w.tolist()):
        if a != b:
            r = col[rp[a]:rp[a + 1]]
            assert r[np.searchsorted(r, b)] == b


# ------------------------------------------------------------------ the widened rows at full size
@pytest.fixture(scope="module")
def rmat18(nk):
    g = nk.graph_generate("rmat", 18, 1)
    n, rp, col = oracle.generate("rmat", 18, 1)
    return g, n, rp, col, nk.autotune(g, 2, 1024)


def test_rmat18_closeness_k1024_full_vector(nk, rmat18):
    g, n, rp, col, opts = rmat18
    far, reach = nk.closeness_sampled(g, 2, 1024, opts)
    src = oracle.sample_sources(n, 2, 1024)
    parts = _slices(lambda p: oracle.closeness_sources(rp, col, p, 1.0), src)
    scale = n / 1024
    assert np.array_equal(far, sum(p[0] for p in parts) * scale)
    assert np.array_equal(reach, sum(p[1] for p in parts) * scale)


def test_rmat18_edge_betweenness_k1024_full_vector(nk, rmat18):
    g, n, rp, col, opts = rmat18
    got = nk.edge_betweenness_sampled(g, 2, 1024, opts)
    src = oracle.sample_sources(n, 2, 1024)
    want = sum(_slices(lambda p: oracle.edge_betweenness_sources(rp, col, p, 1.0), src)) * (n / (2.0 * 1024))
    assert close(got, want)


def test_rmat18_rk_estimate_full_counts(nk, rmat18):
    # the bench leg runs epsilon 0.01; here epsilon 0.03 keeps the oracle's share in seconds
    g, n, rp, col, opts = rmat18
    ro = nk.run_opts(mode=nk.MODE_BATCHED, batch=opts.batch, alpha=opts.alpha)
    got, r, vd = nk.betweenness_rk(g, 0.03, 0.1, 2, ro)
    assert vd == oracle.vertex_diameter_estimate(rp, col) and r == oracle.rk_sample_count(0.03, 0.1, vd)
    cuts = np.linspace(0, r, 17).astype(np.int64)
    counts = sum(_slices(lambda p: sum(oracle.rk_counts(rp, col, 2, int(cuts[i]), int(cuts[i + 1])) for i in p),
                         np.arange(16)))
    assert np.array_equal(got, counts.astype(np.float64) * (n * (n - 1) / (2.0 * r)))


def test_rmat18_weighted_k256_full_vector(nk, rmat18):
    g, n, rp, col, _ = rmat18
    nk.random_weights(g, 5, 16)
    w = oracle.edge_weights(rp, col, 5, 16)
    got = nk.betweenness_weighted_sampled(g, 2, 256)
    src = oracle.sample_sources(n, 2, 256)
    want = sum(_slices(lambda p: oracle.betweenness_weighted_sources(rp, col, w, p, 1.0), src)) * (n / (2.0 * 256))
    assert close(got, want)
