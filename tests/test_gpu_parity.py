"""GPU parity: every step of the CUDA path against the CPU oracle on the same seeded
inputs (through the C ABI).

Bars: distances, path counts, CSR arrays and sampled source sets bit-exact; FP64
scores within 1e-9 relative with a 1e-12 absolute floor.  Every input comes from
tests/graphs.py or from each side's own generator; the oracle never sees a GPU output.
"""
from __future__ import annotations

import numpy as np
import pytest

import graphs as G
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


def both(nk, graph):
    """(gpu graph built from the edge list by the GPU CSR builder, oracle CSR)."""
    n, u, v = graph
    g = nk.graph_from_edges(n, u, v)
    rp, col = oracle.csr_build(n, u, v)
    return g, rp, col


def close(a, b):
    return np.allclose(a, b, rtol=RTOL, atol=ATOL)


MODES = [
    dict(mode=1, tpv=1), dict(mode=1, tpv=4), dict(mode=1, tpv=32),
    dict(mode=1, direction=1), dict(mode=1, direction=2),
    dict(mode=2, batch=64), dict(mode=2, batch=128), dict(mode=2, batch=256),
    dict(mode=2, batch=64, direction=1), dict(mode=2, batch=64, direction=2),
    dict(mode=2, batch=128, alpha=0.05), dict(mode=2, batch=64, alpha=50.0),
    dict(mode=2, batch=128, chunk=64), dict(mode=2, batch=64, direction=2, chunk=32),
]

SMALL = {
    "path": G.path(40), "cycle_odd": G.cycle(31), "cycle_even": G.cycle(30), "star": G.star(50),
    "complete": G.complete(12), "k_ab": G.complete_bipartite(5, 9), "grid": G.grid(9, 13),
    "hypercube": G.hypercube(6), "tree": G.random_tree(300, 3), "gnp": G.gnp(200, 0.04, 5),
    "components": G.disjoint_union(G.path(7), G.gnp(60, 0.1, 2), G.star(5), G.complete(1)),
    "isolated": G.disjoint_union(G.complete(1), G.complete(1), G.path(3)),
    "star_big": G.star(1500),
    "hubs": G.with_hubs(G.disjoint_union(*[G.complete(1)] * 5, G.gnp(1200, 0.004, 9)),
                        [256, 257, 512, 513, 1000], 4),
    "hub_path": G.with_hubs(G.path(700), [600, 300], 5),
}


# ------------------------------------------------------------------ CSR builder
@pytest.mark.parametrize("name", sorted(SMALL))
def test_csr_builder_matches_oracle(nk, name):
    n, u, v = SMALL[name]
    rp, col = oracle.csr_build(n, u, v)
    for graph in ((n, u, v), G.noisy((n, u, v), 1)):
        g = nk.graph_from_edges(*graph)
        grp, gcol = g.export_csr()
        assert np.array_equal(grp, rp) and np.array_equal(gcol, col)
    g = nk.graph_from_csr(rp, col, nk.CSR_VALIDATE)
    assert g.info() == (n, len(col))


def test_csr_canonicalise_and_validate(nk):
    n, u, v = G.gnp(500, 0.02, 8)
    rp, col = oracle.csr_build(n, u, v)
    # one direction only, unsorted, duplicated, with loops: canonicalised on the GPU
    nn, uu, vv = G.noisy((n, u, v), 4)
    order = np.lexsort((vv, uu))
    uu, vv = uu[order], vv[order]
    raw_rp = np.zeros(n + 1, np.int64)
    np.add.at(raw_rp, uu + 1, 1)
    raw_rp = np.cumsum(raw_rp).astype(np.int32)
    g = nk.graph_from_csr(raw_rp, vv, nk.CSR_CANONICALISE)
    grp, gcol = g.export_csr()
    assert np.array_equal(grp, rp) and np.array_equal(gcol, col)
    with pytest.raises(nk.NkError) as e:
        nk.graph_from_csr(raw_rp, vv, nk.CSR_VALIDATE)
    assert e.value.rc == nk.ERR_GRAPH
    bad = col.copy()
    bad[0] = n  # out of range
    with pytest.raises(nk.NkError):
        nk.graph_from_csr(rp, bad, 0)
    with pytest.raises(nk.NkError):
        nk.graph_from_edges(3, np.array([0, 3]), np.array([1, 0]))


def test_csr_long_rows(nk):
    # rows longer than 32 and 4096 use the shared-memory and bitmap sorters
    n = 20000
    rng = np.random.default_rng(3)
    u = np.concatenate([np.zeros(9000, np.int64), np.full(3000, 7), rng.integers(0, n, 5000)])
    v = np.concatenate([rng.integers(0, n, 9000), rng.integers(0, n, 3000), rng.integers(0, n, 5000)])
    rp, col = oracle.csr_build(n, u, v)
    g = nk.graph_from_edges(n, u, v)
    grp, gcol = g.export_csr()
    assert np.array_equal(grp, rp) and np.array_equal(gcol, col)


# ------------------------------------------------------------------ generators
@pytest.mark.parametrize("kind,size,seed,params", [
    ("er", 2000, 1, dict(avg_deg=8.0)), ("er", 1500, 3, dict(avg_deg=20.0)),
    ("er", 7, 2, dict(avg_deg=10.0)), ("er", 1, 1, dict(avg_deg=8.0)),
    ("ba", 5000, 1, dict(m0=8)), ("ba", 3000, 5, dict(m0=1)), ("ba", 1, 1, dict(m0=4)),
    ("rmat", 12, 1, {}), ("rmat", 14, 7, dict(edge_factor=8, a=0.45, b=0.25, c=0.15)),
])
def test_generators_byte_identical(nk, kind, size, seed, params):
    g = nk.graph_generate(kind, size, seed, **params)
    n, rp, col = oracle.generate(kind, size, seed, **params)
    grp, gcol = g.export_csr()
    assert g.n == n
    assert np.array_equal(grp, rp) and np.array_equal(gcol, col)


def test_generators_full_size_configs(nk):
    # R-MAT scale 18 edge factor 16 and BA n = 1e6, m0 = 8: byte-identical CSR
    for kind, size, params in (("rmat", 18, {}), ("ba", 1000000, dict(m0=8))):
        g = nk.graph_generate(kind, size, 1, **params)
        n, rp, col = oracle.generate(kind, size, 1, **params)
        grp, gcol = g.export_csr()
        assert np.array_equal(grp, rp) and np.array_equal(gcol, col), kind
        g.free()


# ------------------------------------------------------------------ sampler
@pytest.mark.parametrize("n,k,seed", [(1, 1, 1), (10, 10, 3), (1000, 1, 2), (5000, 1024, 2),
                                      (262144, 1024, 2), (100000, 99999, 5), (70000, 4096, 0)])
def test_sampler_matches_oracle(nk, n, k, seed):
    assert np.array_equal(nk.sample_sources(n, seed, k), oracle.sample_sources(n, seed, k))


# ------------------------------------------------------------------ forward sweep
@pytest.mark.parametrize("name", sorted(SMALL))
def test_sssp_bit_exact_small(nk, name):
    g, rp, col = both(nk, SMALL[name])
    n = len(rp) - 1
    for s in range(0, n, max(1, n // 25)):
        d, sg = nk.sssp(g, s)
        d0, s0 = oracle.bfs(rp, col, s)
        assert np.array_equal(d, d0) and np.array_equal(sg, s0), (name, s)


def test_sssp_bit_exact_generated(nk):
    for kind, size, params in (("er", 2000, dict(avg_deg=8.0)), ("rmat", 14, {}), ("ba", 20000, dict(m0=4))):
        g = nk.graph_generate(kind, size, 1, **params)
        n, rp, col = oracle.generate(kind, size, 1, **params)
        for s in np.random.default_rng(0).integers(0, n, 12):
            d, sg = nk.sssp(g, int(s))
            d0, s0 = oracle.bfs(rp, col, int(s))
            assert np.array_equal(d, d0) and np.array_equal(sg, s0), (kind, s)


def test_sigma_near_limit_and_overflow(nk):
    g, rp, col = both(nk, G.grid(34, 35))
    d, sg = nk.sssp(g, 0)
    d0, s0 = oracle.bfs(rp, col, 0)
    assert np.array_equal(sg, s0) and int(sg[33 * 35 + 34]) == 14226520737620288370
    g2, _, _ = both(nk, G.grid(35, 35))
    with pytest.raises(nk.NkError) as e:
        nk.sssp(g2, 0)
    assert e.value.rc == nk.ERR_OVERFLOW
    for opts in (nk.run_opts(mode=1), nk.run_opts(mode=2, batch=64)):
        with pytest.raises(nk.NkError) as e:
            nk.betweenness_sources(g2, np.array([0, 1], np.int32), 1.0, opts)
        assert e.value.rc == nk.ERR_OVERFLOW


def _forms(nk):
    return (nk.run_opts(mode=nk.MODE_PER_SOURCE), nk.run_opts(mode=nk.MODE_BATCHED, batch=64),
            nk.run_opts(mode=nk.MODE_BATCHED, batch=256))


def test_scores_with_sigma_near_the_limit(nk):
    # 34 x 35 grid: from a corner sigma reaches C(67, 33) ~ 1.42e19 (2^63.6), where the
    # double-single conversion of sigma and its reciprocal keep about 48 of its 64 bits; the
    # scores of the four corners and a spread of other sources in the per-source form and in
    # batches of 64 and 256
    g, rp, col = both(nk, G.grid(34, 35))
    n = len(rp) - 1
    src = np.array([0, 34, 33 * 35, n - 1] + list(range(1, n - 1, 7)), np.int32)
    _, s0 = oracle.bfs(rp, col, 0)
    assert int(s0.max()) == 14226520737620288370  # C(67, 33) > 2^63
    want = oracle.betweenness_sources(rp, col, src, 1.0)
    for opts in _forms(nk):
        assert close(nk.betweenness_sources(g, src, 1.0, opts), want), opts.mode


def test_scores_on_a_large_hypercube(nk):
    # Q_20 (2^20 vertices, 20 arcs each): sigma from x to its antipode is 20! ~ 2.4e18 (2^61)
    n, u, v = G.hypercube_edges(20)
    g = nk.graph_from_edges(n, u, v)
    rp, col = oracle.csr_build(n, u, v)
    src = np.array([0, n - 1, 0x55555, 0xAAAAA, 12345, 777777, 3, 1 << 19], np.int32)
    _, s0 = oracle.bfs(rp, col, 0)
    assert int(s0[n - 1]) == 2432902008176640000  # 20!
    want = oracle.betweenness_sources(rp, col, src, 1.0)
    for opts in _forms(nk):
        assert close(nk.betweenness_sources(g, src, 1.0, opts), want), opts.mode
    g.free()


# ------------------------------------------------------------------ betweenness
@pytest.mark.parametrize("name", sorted(SMALL))
def test_exact_small_graphs(nk, name):
    g, rp, col = both(nk, SMALL[name])
    want = oracle.betweenness_exact(rp, col)
    assert close(nk.betweenness_exact(g), want)
    n = len(rp) - 1
    src = np.arange(n, dtype=np.int32)
    for m in MODES:
        got = nk.betweenness_sources(g, src, 0.5, nk.run_opts(**m))
        assert close(got, want), (name, m)


def test_exact_er_2000(nk):
    # Erdos-Renyi n = 2000, average degree 8, seed 1, all 2000 sources
    g = nk.graph_generate("er", 2000, 1, avg_deg=8.0)
    n, rp, col = oracle.generate("er", 2000, 1, avg_deg=8.0)
    want = oracle.betweenness_exact(rp, col)
    assert close(nk.betweenness_exact(g), want)
    for m in (dict(mode=1), dict(mode=2, batch=64), dict(mode=2, batch=256)):
        assert close(nk.betweenness_sources(g, np.arange(n, dtype=np.int32), 0.5, nk.run_opts(**m)), want), m


@pytest.mark.parametrize("m", MODES)
def test_sampled_rmat_modes(nk, m):
    g = nk.graph_generate("rmat", 13, 5)
    n, rp, col = oracle.generate("rmat", 13, 5)
    k = 333  # not a multiple of any batch size
    want = oracle.betweenness_sampled(rp, col, 4, k)
    got = nk.betweenness_sampled(g, 4, k, nk.run_opts(**m))
    assert close(got, want), m


def test_per_source_push_levels(nk):
    # sources whose sweep has a level l >= 1 with 4 * arcs(l + 1) < arcs(l) and a hub (more
    # than 256 arcs) on it: the per-source backward pushes psi into that level's light
    # vertices and pulls for its hubs
    g = nk.graph_generate("rmat", 14, 3)
    n, rp, col = oracle.generate("rmat", 14, 3)
    deg = np.diff(rp)
    picked = []
    for s in oracle.sample_sources(n, 6, 400):
        if deg[s] == 0:
            continue
        d, _ = oracle.bfs(rp, col, int(s))
        arcs = np.bincount(d[d >= 0], weights=deg[d >= 0])
        hubs = np.bincount(d[(d >= 0) & (deg > 256)], minlength=len(arcs))
        if any(4 * arcs[l + 1] < arcs[l] and hubs[l] > 0 for l in range(1, len(arcs) - 1)):
            picked.append(int(s))
        if len(picked) == 24:
            break
    assert len(picked) == 24
    src = np.array(picked, dtype=np.int32)
    want = oracle.betweenness_sources(rp, col, src, 0.5)
    assert close(nk.betweenness_sources(g, src, 0.5, nk.run_opts(mode=1)), want)
    assert close(nk.betweenness_sources(g, src, 0.5, nk.run_opts(mode=1, direction=1)), want)
    want_e = oracle.edge_betweenness_sampled(rp, col, 6, 400)   # the whole sample they come from
    assert close(nk.edge_betweenness_sampled(g, 6, 400, nk.run_opts(mode=1)), want_e)


def test_sampled_ba_and_isolated_sources(nk):
    # R-MAT leaves many isolated vertices: sampled sources that are isolated count
    g = nk.graph_generate("rmat", 11, 9, edge_factor=2)
    n, rp, col = oracle.generate("rmat", 11, 9, edge_factor=2)
    assert np.any(np.diff(rp)[oracle.sample_sources(n, 1, 500)] == 0)
    assert close(nk.betweenness_sampled(g, 1, 500), oracle.betweenness_sampled(rp, col, 1, 500))
    g = nk.graph_generate("ba", 30000, 2, m0=8)
    n, rp, col = oracle.generate("ba", 30000, 2, m0=8)
    assert close(nk.betweenness_sampled(g, 3, 200), oracle.betweenness_sampled(rp, col, 3, 200))


def test_sampled_k_equals_n_is_exact(nk):
    g, rp, col = both(nk, G.gnp(150, 0.05, 12))
    assert close(nk.betweenness_sampled(g, 77, 150), oracle.betweenness_exact(rp, col))


def test_deep_graph_falls_back_to_per_source(nk):
    # a path of 3000 vertices is deeper than the batched form's level slabs
    g, rp, col = both(nk, G.path(3000))
    src = np.array([0, 5, 1499, 2999], np.int32)
    want = oracle.betweenness_sources(rp, col, src, 1.0)
    got = nk.betweenness_sources(g, src, 1.0, nk.run_opts(mode=2, batch=64))
    assert close(got, want)


def test_device_pointer_outputs(nk):
    import torch
    g = nk.graph_generate("ba", 4000, 3, m0=4)
    n, rp, col = oracle.generate("ba", 4000, 3, m0=4)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    nk.betweenness_sampled(g, 5, 100, nk.run_opts(mode=2), out=out)
    assert close(out.cpu().numpy(), oracle.betweenness_sampled(rp, col, 5, 100))
    src = torch.from_numpy(oracle.sample_sources(n, 5, 100)).cuda()
    out2 = torch.empty(n, dtype=torch.float64, device="cuda")
    nk.betweenness_sources(g, src, n / 200.0, nk.run_opts(mode=1), out=out2)
    assert close(out2.cpu().numpy(), out.cpu().numpy())


def test_argument_errors(nk):
    g = nk.graph_generate("er", 100, 1, avg_deg=4.0)
    for k in (0, 101):
        with pytest.raises(nk.NkError) as e:
            nk.betweenness_sampled(g, 1, k)
        assert e.value.rc == nk.ERR_ARG
    with pytest.raises(nk.NkError):
        nk.sssp(g, 100)
    with pytest.raises(nk.NkError):
        nk.betweenness_sources(g, np.array([0, 100], np.int32), 1.0)
    with pytest.raises(nk.NkError):
        nk.betweenness_sampled(g, 1, 10, nk.run_opts(mode=2, batch=96))


def test_bounded_wait_times_out_cleanly(nk):
    assert nk.selftest_wait_timeout(50_000_000) == nk.ERR_TIMEOUT
    g = nk.graph_generate("er", 200, 2, avg_deg=5.0)
    n, rp, col = oracle.generate("er", 200, 2, avg_deg=5.0)
    assert close(nk.betweenness_exact(g), oracle.betweenness_exact(rp, col))


def test_autotune_then_run(nk):
    g = nk.graph_generate("rmat", 12, 3)
    n, rp, col = oracle.generate("rmat", 12, 3)
    best = nk.autotune(g, 2, 300)
    assert best.batch in (64, 128, 256) and best.alpha > 0
    assert close(nk.betweenness_sampled(g, 2, 300), oracle.betweenness_sampled(rp, col, 2, 300))


def test_cuda_graph_capture_and_replay(nk):
    # NK_RUN_CUDA_GRAPH: the first call captures, later identical calls replay; every
    # replay recomputes the same result, a changed seed recaptures; kernels are counted
    import torch
    g = nk.graph_generate("rmat", 13, 8)
    n, rp, col = oracle.generate("rmat", 13, 8)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    flags = nk.RUN_CUDA_GRAPH
    for seed in (3, 3, 4, 4, 3):
        out.fill_(-1.0)
        l0 = nk.launch_count()
        nk.betweenness_sampled(g, seed, 300, nk.run_opts(mode=2, batch=128, flags=flags), out=out)
        assert nk.launch_count() > l0
        assert close(out.cpu().numpy(), oracle.betweenness_sampled(rp, col, seed, 300)), seed
    # a graph deeper than the captured level slabs falls back to the regular path
    gp, rpp, colp = both(nk, G.path(400))
    outp = torch.empty(400, dtype=torch.float64, device="cuda")
    nk.betweenness_sampled(gp, 2, 100, nk.run_opts(mode=2, batch=64, flags=flags), out=outp)
    assert close(outp.cpu().numpy(), oracle.betweenness_sampled(rpp, colp, 2, 100))


# ------------------------------------------------------------------ closeness (Table 1)
@pytest.mark.parametrize("name", ["path", "star", "cycle_odd", "grid", "components", "hubs", "tree"])
def test_closeness_exact_small(nk, name):
    g, rp, col = both(nk, SMALL[name])
    far0, reach0 = oracle.closeness_exact(rp, col)
    far, reach = nk.closeness_exact(g)
    assert np.array_equal(far, far0) and np.array_equal(reach, reach0)
    n = len(rp) - 1
    for m in (dict(mode=1), dict(mode=2, batch=64, direction=1), dict(mode=2, batch=256, direction=2)):
        f2, r2 = nk.closeness_sampled(g, 5, n, nk.run_opts(**m))
        assert np.array_equal(f2, far0) and np.array_equal(r2, reach0), m


def test_closeness_sampled_generated(nk):
    for kind, size, params, k in (("rmat", 14, {}, 500), ("ba", 50000, dict(m0=4), 300)):
        g = nk.graph_generate(kind, size, 3, **params)
        n, rp, col = oracle.generate(kind, size, 3, **params)
        f0, r0 = oracle.closeness_sampled(rp, col, 9, k)
        f1, r1 = nk.closeness_sampled(g, 9, k)
        assert np.array_equal(f1, f0) and np.array_equal(r1, r0), kind
    gp, rpp, colp = both(nk, G.path(3000))   # deeper than the level slabs: per-source fallback
    f0, r0 = oracle.closeness_sampled(rpp, colp, 4, 70)
    f1, r1 = nk.closeness_sampled(gp, 4, 70, nk.run_opts(mode=2, batch=64))
    assert np.array_equal(f1, f0) and np.array_equal(r1, r0)


def test_closeness_with_path_count_overflow(nk):
    # 35 x 35 grid: corner-to-corner path counts exceed 2^64 - 1; distances are unaffected,
    # so closeness succeeds in every form (batched sweeps rerun such batches per source)
    g, rp, col = both(nk, G.grid(35, 35))
    far0, reach0 = oracle.closeness_exact(rp, col)
    for m in (dict(mode=1), dict(mode=2, batch=64), dict(mode=2, batch=128, direction=2)):
        f, r = nk.closeness_sampled(g, 1, len(rp) - 1, nk.run_opts(**m))
        assert np.array_equal(f, far0) and np.array_equal(r, reach0), m


def test_closeness_device_outputs(nk):
    import torch
    g = nk.graph_generate("rmat", 13, 2)
    n, rp, col = oracle.generate("rmat", 13, 2)
    f0, r0 = oracle.closeness_sampled(rp, col, 6, 200)
    far = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    reach = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    nk.closeness_sampled(g, 6, 200, nk.run_opts(mode=2, batch=128), out=(far, reach))
    assert np.array_equal(far.cpu().numpy(), f0) and np.array_equal(reach.cpu().numpy(), r0)


# ------------------------------------------------------------------ edge betweenness (Section 4.3)
@pytest.mark.parametrize("name", ["path", "star", "cycle_even", "k_ab", "grid", "tree", "components",
                                  "isolated", "hubs", "hub_path", "star_big"])
def test_edge_betweenness_exact_small(nk, name):
    g, rp, col = both(nk, SMALL[name])
    want = oracle.edge_betweenness_exact(rp, col)
    assert close(nk.edge_betweenness_exact(g), want)
    n = len(rp) - 1
    for m in MODES:
        got = nk.edge_betweenness_sampled(g, 3, n, nk.run_opts(**m))
        assert close(got, want), (name, m)


def test_edge_betweenness_sampled_generated(nk):
    for kind, size, params, k in (("rmat", 13, {}, 300), ("ba", 20000, dict(m0=4), 200),
                                  ("er", 2000, dict(avg_deg=8.0), 2000)):
        g = nk.graph_generate(kind, size, 5, **params)
        n, rp, col = oracle.generate(kind, size, 5, **params)
        want = oracle.edge_betweenness_sampled(rp, col, 8, k)
        for m in (dict(), dict(mode=2, batch=128), dict(mode=1)):
            assert close(nk.edge_betweenness_sampled(g, 8, k, nk.run_opts(**m)), want), (kind, m)


def test_edge_betweenness_deep_and_overflow(nk):
    gp, rp, col = both(nk, G.path(3000))   # deeper than the level slabs: per-source fallback
    want = oracle.edge_betweenness_sampled(rp, col, 4, 70)
    assert close(nk.edge_betweenness_sampled(gp, 4, 70, nk.run_opts(mode=2, batch=64)), want)
    g2, _, _ = both(nk, G.grid(35, 35))
    for opts in (nk.run_opts(mode=1), nk.run_opts(mode=2, batch=64)):
        with pytest.raises(nk.NkError) as e:
            nk.edge_betweenness_sampled(g2, 1, 1225, opts)
        assert e.value.rc == nk.ERR_OVERFLOW


def test_edge_betweenness_device_output(nk):
    import torch
    g = nk.graph_generate("rmat", 12, 7)
    n, rp, col = oracle.generate("rmat", 12, 7)
    want = oracle.edge_betweenness_sampled(rp, col, 2, 256)
    out = torch.full((len(col),), -1.0, dtype=torch.float64, device="cuda")
    nk.edge_betweenness_sampled(g, 2, 256, nk.run_opts(mode=2, batch=256), out=out)
    assert close(out.cpu().numpy(), want)


# ------------------------------------------------------------------ error-bounded estimate (Section 3.2)
RK_MODES = [dict(), dict(mode=1), dict(mode=1, direction=2), dict(mode=2, batch=64, direction=1),
            dict(mode=2, batch=128, direction=2), dict(mode=2, batch=256)]


@pytest.mark.parametrize("name", ["path", "grid", "tree", "components", "isolated", "complete",
                                  "hubs", "star_big", "hub_path"])
def test_rk_small_graphs(nk, name):
    g, rp, col = both(nk, SMALL[name])
    assert nk.vertex_diameter_estimate(g) == oracle.vertex_diameter_estimate(rp, col)
    want, r0, vd0 = oracle.betweenness_rk(rp, col, 0.1, 0.1, 7)
    for m in RK_MODES:
        got, r, vd = nk.betweenness_rk(g, 0.1, 0.1, 7, nk.run_opts(**m))
        assert (r, vd) == (r0, vd0)
        assert np.array_equal(got, want), (name, m)


def test_rk_generated(nk):
    for kind, size, params, eps in (("rmat", 13, {}, 0.05), ("ba", 20000, dict(m0=4), 0.08),
                                    ("er", 2000, dict(avg_deg=8.0), 0.05)):
        g = nk.graph_generate(kind, size, 9, **params)
        n, rp, col = oracle.generate(kind, size, 9, **params)
        want, r0, vd0 = oracle.betweenness_rk(rp, col, eps, 0.1, 21)
        for m in (dict(), dict(mode=2, batch=128), dict(mode=1)):
            got, r, vd = nk.betweenness_rk(g, eps, 0.1, 21, nk.run_opts(**m))
            assert (r, vd) == (r0, vd0) and np.array_equal(got, want), (kind, m)


def test_rk_deep_overflow_and_errors(nk):
    gp, rp, col = both(nk, G.path(3000))   # deeper than the level slabs: per-source fallback
    want, r0, _ = oracle.betweenness_rk(rp, col, 0.3, 0.1, 5)
    got, r, vd = nk.betweenness_rk(gp, 0.3, 0.1, 5, nk.run_opts(mode=2, batch=64))
    assert r == r0 and vd == 3000 and np.array_equal(got, want)
    g2, rp2, col2 = both(nk, G.grid(35, 35))
    seeds = []                                     # the oracle says which seeds overflow
    for sd in range(12):
        try:
            oracle.betweenness_rk(rp2, col2, 0.1, 0.1, sd)
            seeds.append((sd, False))
        except oracle.OracleError as eo:
            assert eo.rc == oracle.ERR_OVERFLOW    # a sampled source near a corner
            seeds.append((sd, True))
    assert any(o for _, o in seeds) and not all(o for _, o in seeds)
    for sd, overflows in seeds[:6]:
        for opts in (nk.run_opts(mode=1), nk.run_opts(mode=2, batch=64)):
            if overflows:
                with pytest.raises(nk.NkError) as e:
                    nk.betweenness_rk(g2, 0.1, 0.1, sd, opts)
                assert e.value.rc == nk.ERR_OVERFLOW
            else:
                got, _, _ = nk.betweenness_rk(g2, 0.1, 0.1, sd, opts)
                assert np.array_equal(got, oracle.betweenness_rk(rp2, col2, 0.1, 0.1, sd)[0])
    for eps, delta in ((0.0, 0.1), (1.0, 0.1), (0.1, 0.0), (0.1, 1.5)):
        with pytest.raises(nk.NkError) as e:
            nk.betweenness_rk(gp, eps, delta, 1)
        assert e.value.rc == nk.ERR_ARG


def test_rk_device_output(nk):
    import torch
    g = nk.graph_generate("rmat", 12, 3)
    n, rp, col = oracle.generate("rmat", 12, 3)
    want, r0, _ = oracle.betweenness_rk(rp, col, 0.07, 0.05, 4)
    out = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    _, r, _ = nk.betweenness_rk(g, 0.07, 0.05, 4, nk.run_opts(mode=2, batch=256), out=out)
    assert r == r0 and np.array_equal(out.cpu().numpy(), want)


# ------------------------------------------------------------------ weighted graphs (Sections 2.3, 3.4)
def weighted_both(nk, graph, seed, wmax):
    g, rp, col = both(nk, graph)
    nk.random_weights(g, seed, wmax)
    return g, rp, col, oracle.edge_weights(rp, col, seed, wmax)


def test_weights_generated_identically_and_checked(nk):
    g, rp, col, w = weighted_both(nk, G.gnp(300, 0.03, 1), 5, 9)
    assert np.array_equal(nk.export_weights(g), w)
    nk.set_weights(g, w)
    assert np.array_equal(nk.export_weights(g), w)
    for bad in (w + np.eye(1, len(w), 0, dtype=np.int32)[0], np.zeros_like(w)):
        with pytest.raises(nk.NkError) as e:
            nk.set_weights(g, bad)
        assert e.value.rc == nk.ERR_GRAPH
    g2, _, _ = both(nk, G.path(10))
    with pytest.raises(nk.NkError) as e:
        nk.betweenness_weighted_exact(g2)
    assert e.value.rc == nk.ERR_ARG


@pytest.mark.parametrize("name", ["path", "cycle_even", "k_ab", "grid", "hypercube", "tree", "gnp",
                                  "components", "isolated", "hubs", "hub_path"])
def test_weighted_exact_small(nk, name):
    for wmax in (1, 3, 50):
        g, rp, col, w = weighted_both(nk, SMALL[name], 7 + wmax, wmax)
        n = len(rp) - 1
        assert close(nk.betweenness_weighted_exact(g), oracle.betweenness_weighted_exact(rp, col, w)), wmax
        for s in sorted({0, n // 3, n - 1}):
            d, sg = nk.sssp_weighted(g, s)
            d0, s0 = oracle.sssp_weighted(rp, col, w, s)
            assert np.array_equal(d, d0) and np.array_equal(sg, s0), (wmax, s)


def test_weighted_sampled_generated(nk):
    for kind, size, params, wmax, k in (("rmat", 12, {}, 16, 100), ("ba", 5000, dict(m0=4), 5, 64),
                                        ("er", 2000, dict(avg_deg=8.0), 100, 50)):
        g = nk.graph_generate(kind, size, 4, **params)
        n, rp, col = oracle.generate(kind, size, 4, **params)
        nk.random_weights(g, 12, wmax)
        w = oracle.edge_weights(rp, col, 12, wmax)
        want = oracle.betweenness_weighted_sampled(rp, col, w, 6, k)
        assert close(nk.betweenness_weighted_sampled(g, 6, k), want), kind


def test_weighted_overflow_and_device_output(nk):
    import torch
    g, rp, col, w = weighted_both(nk, G.grid(35, 35), 1, 1)
    with pytest.raises(nk.NkError) as e:
        nk.sssp_weighted(g, 0)
    assert e.value.rc == nk.ERR_OVERFLOW
    g, rp, col, w = weighted_both(nk, G.gnp(500, 0.02, 3), 2, 20)
    want = oracle.betweenness_weighted_sampled(rp, col, w, 3, 40)
    out = torch.full((500,), -1.0, dtype=torch.float64, device="cuda")
    nk.betweenness_weighted_sampled(g, 3, 40, None, out=out)
    assert close(out.cpu().numpy(), want)


# ------------------------------------------------------------------ degenerate inputs of the widened rows
@pytest.mark.parametrize("graph", [G.complete(1), G.disjoint_union(G.complete(1), G.complete(1), G.complete(1)),
                                   G.path(2), G.star(3)])
def test_widened_rows_on_degenerate_graphs(nk, graph):
    g, rp, col = both(nk, graph)
    n = len(rp) - 1
    f0, r0 = oracle.closeness_exact(rp, col)
    f1, r1 = nk.closeness_exact(g)
    assert np.array_equal(f1, f0) and np.array_equal(r1, r0)
    e = nk.edge_betweenness_exact(g)
    assert len(e) == len(col) and close(e, oracle.edge_betweenness_exact(rp, col))
    for m in (dict(mode=1), dict(mode=2, batch=64)):
        assert close(nk.edge_betweenness_sampled(g, 1, n, nk.run_opts(**m)), oracle.edge_betweenness_exact(rp, col))
    want, r, vd = oracle.betweenness_rk(rp, col, 0.3, 0.3, 2)
    got, r1_, vd1 = nk.betweenness_rk(g, 0.3, 0.3, 2)
    assert (r1_, vd1) == (r, vd) and np.array_equal(got, want)
    nk.random_weights(g, 3, 4)
    w = oracle.edge_weights(rp, col, 3, 4)
    assert close(nk.betweenness_weighted_exact(g), oracle.betweenness_weighted_exact(rp, col, w))
    d, sg = nk.sssp_weighted(g, n - 1)
    d0, s0 = oracle.sssp_weighted(rp, col, w, n - 1)
    assert np.array_equal(d, d0) and np.array_equal(sg, s0)


def test_grid_ctas_option_parity_and_determinism(nk):
    g, rp, col, w = weighted_both(nk, SMALL["hubs"], 11, 6)
    n = len(rp) - 1
    want = oracle.betweenness_weighted_sampled(rp, col, w, 3, 300)
    runs = [nk.betweenness_weighted_sampled(g, 3, 300, nk.run_opts(grid_ctas=gc)) for gc in (0, 0, 1, 7, 40)]
    assert np.array_equal(runs[0], runs[1])          # the same groups sum in the same order
    for r in runs:
        assert close(r, want)
    vb = oracle.betweenness_sampled(rp, col, 3, 300)
    for m in (dict(mode=1, grid_ctas=5), dict(mode=2, batch=64, grid_ctas=9), dict(mode=2, batch=256, grid_ctas=2)):
        assert close(nk.betweenness_sampled(g, 3, 300, nk.run_opts(**m)), vb), m
    with pytest.raises(nk.NkError) as e:
        nk.betweenness_sampled(g, 3, 300, nk.run_opts(grid_ctas=-1))
    assert e.value.rc == nk.ERR_ARG


def test_chunk_option(nk):
    g, rp, col = both(nk, SMALL["hubs"])
    want = oracle.betweenness_sampled(rp, col, 4, 500)
    for chunk in (32, 96, 128, 512, 4096):
        for B in (64, 256):
            assert close(nk.betweenness_sampled(g, 4, 500, nk.run_opts(mode=2, batch=B, chunk=chunk)), want), (chunk, B)
    for bad in (-32, 16, 100, 8192):
        with pytest.raises(nk.NkError) as e:
            nk.betweenness_sampled(g, 4, 500, nk.run_opts(mode=2, chunk=bad))
        assert e.value.rc == nk.ERR_ARG
    opts = nk.autotune(g, 4, 500)
    assert opts.chunk in (0, 128)
    assert close(nk.betweenness_sampled(g, 4, 500, opts), want)


# ------------------------------------------------------------------ relabelled copy of the graph
@pytest.mark.parametrize("name", ["hubs", "components", "grid", "star_big", "path"])
def test_relabel_parity(nk, name):
    g, rp, col = both(nk, SMALL[name])
    n = len(rp) - 1
    want = oracle.betweenness_exact(rp, col)
    for m in (dict(mode=2, batch=64), dict(mode=2, batch=128, direction=2), dict(mode=2, batch=256, chunk=64)):
        got = nk.betweenness_sources(g, np.arange(n, dtype=np.int32), 0.5, nk.run_opts(flags=nk.RUN_RELABEL, **m))
        assert close(got, want), (name, m)


@pytest.mark.parametrize("name", ["hubs", "components", "grid", "star_big"])
def test_relabel_edge_parity(nk, name):
    # per-arc sums indexed by the copy's arcs, read back per caller arc (both directions)
    g, rp, col = both(nk, SMALL[name])
    n = len(rp) - 1
    want = oracle.edge_betweenness_exact(rp, col)
    for m in (dict(mode=2, batch=64), dict(mode=2, batch=128, direction=2), dict(mode=2, batch=256, chunk=64)):
        got = nk.edge_betweenness_sampled(g, 3, n, nk.run_opts(flags=nk.RUN_RELABEL, **m))
        assert close(got, want), (name, m)


def test_relabel_edge_sampled_generated(nk):
    import torch
    g = nk.graph_generate("rmat", 13, 5)
    n, rp, col = oracle.generate("rmat", 13, 5)
    want = oracle.edge_betweenness_sampled(rp, col, 8, 300)
    o = nk.run_opts(mode=2, batch=256, alpha=16.0, flags=nk.RUN_RELABEL)
    assert close(nk.edge_betweenness_sampled(g, 8, 300, o), want)
    out = torch.full((len(col),), -1.0, dtype=torch.float64, device="cuda")
    nk.edge_betweenness_sampled(g, 8, 300, o, out=out)
    assert close(out.cpu().numpy(), want)


def test_relabel_sampled_device_graph_and_autotune(nk):
    import torch
    g = nk.graph_generate("rmat", 14, 3)
    n, rp, col = oracle.generate("rmat", 14, 3)
    want = oracle.betweenness_sampled(rp, col, 5, 300)
    o = nk.run_opts(mode=2, batch=128, alpha=16.0, flags=nk.RUN_RELABEL)
    assert close(nk.betweenness_sampled(g, 5, 300, o), want)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    go = nk.run_opts(mode=2, batch=128, alpha=16.0, flags=nk.RUN_RELABEL | nk.RUN_CUDA_GRAPH)
    for _ in range(2):                                  # capture, then replay
        out.fill_(-1.0)
        nk.betweenness_sampled(g, 5, 300, go, out=out)
        assert close(out.cpu().numpy(), want)
    opts = nk.autotune(g, 5, 300)
    assert opts.flags & (nk.RUN_RELABEL | nk.RUN_NO_RELABEL)
    assert close(nk.betweenness_sampled(g, 5, 300, opts), want)
    assert close(nk.betweenness_sampled(g, 5, 300), want)   # the tuned choice, no options


def test_sharded_helper_on_one_rank(nk):
    # the GPU form of the split over ranks (sampler on the device, the rank's slice through
    # nk_betweenness_sources, scale n/(2k)) in a one-rank NCCL group equals the plain call
    import os
    import socket
    import torch
    import torch.distributed as dist
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1)
    try:
        g = nk.graph_generate("rmat", 14, 5)
        n = g.n
        got = nk.betweenness_sampled_sharded(g, 9, 300, nk.run_opts(mode=nk.MODE_BATCHED, batch=64))
        want = nk.betweenness_sampled(g, 9, 300, nk.run_opts(mode=nk.MODE_BATCHED, batch=64))
        assert got.is_cuda and got.numel() == n
        assert close(got.cpu().numpy(), want)
        g.free()
    finally:
        dist.destroy_process_group()
