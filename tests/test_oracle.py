"""Pins for the CPU oracle: closed forms, brute force, invariants and published values.

These tests check the oracle against things other than itself (the paper's definition
of betweenness written as closed forms, an independent brute-force enumeration,
mathematical invariants, published generator outputs), so that a dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one of them.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest

import graphs as G
import oracle
from bruteforce import betweenness_bruteforce, floyd_warshall, sssp_bruteforce

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csr(graph):
    n, u, v = graph
    rp, col = oracle.csr_build(n, u, v)
    return n, rp, col


def exact(graph):
    n, rp, col = csr(graph)
    return oracle.betweenness_exact(rp, col)


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    return rows


# ------------------------------------------------------------------ random numbers
def test_splitmix64_published_vectors():
    want = [r[0] for r in read_golden("splitmix64_seed1234567.txt")]
    got = [oracle.stream(1234567, i) for i in range(5)]
    assert got == want


def test_log_series_matches_libm():
    xs = np.concatenate([np.linspace(2.0 ** -53, 1.0, 4001),
                         1.0 - np.arange(1, 2000) * 2.0 ** -53,
                         2.0 ** -np.arange(0, 53, dtype=np.float64)])
    for x in xs:
        got, want = oracle.log(float(x)), math.log(float(x))
        assert abs(got - want) <= 4 * np.spacing(abs(want)) + 1e-300, (x, got, want)
    assert oracle.log(1.0) == 0.0


# ------------------------------------------------------------------ CSR builder
def test_csr_canonical_form():
    g = G.gnp(40, 0.2, 7)
    n, rp, col = csr(g)
    _, rp2, col2 = csr(G.noisy(g, 3))
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    adj = set()
    for x in range(n):
        row = col[rp[x]:rp[x + 1]]
        assert np.all(np.diff(row) > 0)          # sorted, no duplicates
        assert x not in row                      # no self-loops
        adj.update((x, int(y)) for y in row)
    assert all((y, x) in adj for x, y in adj)  # symmetric
    assert len(adj) == 2 * len({(min(a, b), max(a, b)) for a, b in zip(g[1], g[2])})


def test_csr_rejects_out_of_range():
    with pytest.raises(oracle.OracleError):
        oracle.csr_build(3, np.array([0, 3], np.int32), np.array([1, 0], np.int32))


# ------------------------------------------------------------------ distances
@pytest.mark.parametrize("graph", [G.path(9), G.cycle(10), G.cycle(11), G.grid(4, 6),
                                   G.gnp(30, 0.1, 1), G.gnp(64, 0.05, 2),
                                   G.disjoint_union(G.path(5), G.star(6), G.complete(4))])
def test_bfs_distances_match_floyd_warshall(graph):
    n, rp, col = csr(graph)
    d = floyd_warshall(*graph)
    for s in range(n):
        dist, _ = oracle.bfs(rp, col, s)
        assert np.array_equal(dist, d[s])


def test_distance_closed_forms():
    n, rp, col = csr(G.cycle(13))
    for s in (0, 5):
        dist, sigma = oracle.bfs(rp, col, s)
        j = np.arange(n)
        assert np.array_equal(dist, np.minimum(np.abs(j - s), n - np.abs(j - s)))
        assert np.all(sigma == 1)  # odd cycle: unique shortest paths
    n, rp, col = csr(G.cycle(12))
    dist, sigma = oracle.bfs(rp, col, 0)
    assert sigma[6] == 2 and np.all(np.delete(sigma, 6) == 1)


# ------------------------------------------------------------------ path counts
def test_sigma_grid_binomials():
    rows, cols = 7, 9
    n, rp, col = csr(G.grid(rows, cols))
    dist, sigma = oracle.bfs(rp, col, 0)
    for i in range(rows):
        for j in range(cols):
            assert dist[i * cols + j] == i + j
            assert int(sigma[i * cols + j]) == comb(i + j, i)


def test_sigma_near_uint64_limit_and_overflow():
    gold = {(i, j): s for i, j, s in read_golden("binomial_grid_sigma.txt")}
    n, rp, col = csr(G.grid(34, 35))
    _, sigma = oracle.bfs(rp, col, 0)
    assert int(sigma[33 * 35 + 33]) == gold[(33, 33)]
    assert int(sigma[33 * 35 + 34]) == gold[(33, 34)]
    assert gold[(34, 34)] >= 2 ** 64
    n, rp, col = csr(G.grid(35, 35))
    with pytest.raises(oracle.OracleError) as e:
        oracle.bfs(rp, col, 0)
    assert e.value.rc == oracle.ERR_OVERFLOW


def test_sigma_hypercube_factorials():
    d = 6
    n, rp, col = csr(G.hypercube(d))
    dist, sigma = oracle.bfs(rp, col, 0)
    for x in range(n):
        pc = bin(x).count("1")
        assert dist[x] == pc and int(sigma[x]) == factorial(pc)


def test_sigma_trees_and_bipartite():
    n, rp, col = csr(G.random_tree(200, 5))
    for s in (0, 17, 199):
        dist, sigma = oracle.bfs(rp, col, s)
        assert np.all(sigma == 1) and np.all(dist >= 0)
    a, b = 4, 7
    n, rp, col = csr(G.complete_bipartite(a, b))
    dist, sigma = oracle.bfs(rp, col, 0)           # from side A
    assert np.all(sigma[1:a] == b) and np.all(dist[1:a] == 2)
    dist, sigma = oracle.bfs(rp, col, a)           # from side B
    assert np.all(sigma[a + 1:] == a) and np.all(dist[a + 1:] == 2)


@pytest.mark.parametrize("seed", range(6))
def test_sssp_bruteforce_small(seed):
    g = G.gnp(10, 0.3 + 0.05 * seed, 100 + seed)
    n, rp, col = csr(g)
    for s in range(n):
        dist, sigma = oracle.bfs(rp, col, s)
        bd, bs = sssp_bruteforce(*g, s)
        assert np.array_equal(dist, bd)
        assert [int(x) for x in sigma] == [int(x) for x in bs]


# ------------------------------------------------------------------ betweenness closed forms
@pytest.mark.parametrize("n", [2, 3, 8, 31])
def test_path(n):
    c = exact(G.path(n))
    i = np.arange(n)
    assert np.array_equal(c, (i * (n - 1 - i)).astype(float))


@pytest.mark.parametrize("n", [3, 4, 25])
def test_star(n):
    c = exact(G.star(n))
    assert c[0] == (n - 1) * (n - 2) / 2 and np.all(c[1:] == 0)


@pytest.mark.parametrize("n", [5, 7, 12, 20, 21])
def test_cycle(n):
    c = exact(G.cycle(n))
    r = n // 2
    want = r * (r - 1) / 2 if n % 2 else (r - 1) ** 2 / 2
    assert np.allclose(c, want, rtol=1e-13, atol=0)


def test_complete_and_bipartite():
    assert np.all(exact(G.complete(9)) == 0)
    a, b = 3, 5
    c = exact(G.complete_bipartite(a, b))
    assert np.allclose(c[:a], comb(b, 2) / a, rtol=1e-14)
    assert np.allclose(c[a:], comb(a, 2) / b, rtol=1e-14)


def test_hypercube_q4():
    c = exact(G.hypercube(4))
    assert np.allclose(c, 8.5, rtol=1e-14)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_trees_component_formula(seed):
    n = 300
    g = G.random_tree(n, seed)
    c = exact(g)
    adj = [[] for _ in range(n)]
    for a, b in zip(g[1].tolist(), g[2].tolist()):
        adj[a].append(b)
        adj[b].append(a)
    # c(v) = [(n-1)^2 - sum_i s_i^2] / 2 over the components of T - v
    for v in range(0, n, 7):
        sizes = []
        for start in adj[v]:
            seen, stack = {v, start}, [start]
            while stack:
                x = stack.pop()
                for y in adj[x]:
                    if y not in seen:
                        seen.add(y)
                        stack.append(y)
            sizes.append(len(seen) - 1)
        assert c[v] == ((n - 1) ** 2 - sum(s * s for s in sizes)) / 2


# ------------------------------------------------------------------ brute force on tiny graphs
def _close(c, ref):
    ref = np.array([float(x) for x in ref])
    return np.allclose(c, ref, rtol=1e-12, atol=1e-12)


def test_all_labelled_graphs_on_5_vertices():
    for mask in range(1 << 10):
        g = G.from_mask(5, mask)
        assert _close(exact(g), betweenness_bruteforce(*g)), mask


@pytest.mark.parametrize("seed", range(40))
def test_random_small_graphs_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(6, 13))
    kind = seed % 4
    if kind == 0:
        g = G.gnp(n, float(rng.uniform(0.15, 0.5)), seed)
    elif kind == 1:
        g = G.random_tree(n, seed)
    elif kind == 2:
        g = G.gnp(n, 0.85, seed)                                # near-complete
    else:
        g = G.disjoint_union(G.gnp(n // 2, 0.5, seed), G.gnp(n - n // 2, 0.4, seed + 1))
    assert _close(exact(g), betweenness_bruteforce(*g))


def test_single_source_dependencies_bruteforce():
    # delta_s(v) = sum_t sigma_st(v)/sigma_st, checked one source at a time.
    from bruteforce import adjacency, enumerate_shortest_paths
    g = G.gnp(11, 0.35, 9)
    n, rp, col = csr(g)
    adj = adjacency(*g)
    for s in range(n):
        delta = oracle.dependencies(rp, col, s)
        ref = [Fraction(0)] * n
        for t in range(n):
            if t == s:
                continue
            ps = enumerate_shortest_paths(adj, s, t)
            for p in ps:
                for x in p[1:-1]:
                    ref[x] += Fraction(1, len(ps))
        ref[s] = delta[s]  # delta_s(s) is not a betweenness term
        assert _close(delta, ref)


# ------------------------------------------------------------------ invariant
def pair_distance_sum(n, rp, col):
    tot = 0
    for s in range(n):
        dist, _ = oracle.bfs(rp, col, s)
        r = dist[dist > 0]
        tot += int(np.sum(r - 1))
    return tot / 2


@pytest.mark.parametrize("graph", [G.gnp(120, 0.05, 4), G.grid(9, 13), G.random_tree(150, 8),
                                   G.disjoint_union(G.cycle(30), G.gnp(60, 0.1, 5), G.star(9))])
def test_sum_invariant(graph):
    n, rp, col = csr(graph)
    c = oracle.betweenness_exact(rp, col)
    want = pair_distance_sum(n, rp, col)
    assert math.isclose(c.sum(), want, rel_tol=1e-12)


def test_sum_invariant_generated_er():
    n, rp, col = oracle.generate("er", 600, 11, avg_deg=6.0)
    c = oracle.betweenness_exact(rp, col)
    assert math.isclose(c.sum(), pair_distance_sum(n, rp, col), rel_tol=1e-12)


# ------------------------------------------------------------------ sampler and sampled estimate
def test_sampler_properties():
    n, k = 5000, 300
    src = oracle.sample_sources(n, 2, k)
    assert len(src) == k and np.all(np.diff(src) > 0) and src[0] >= 0 and src[-1] < n
    keys = np.array([oracle.stream(2, v) for v in range(n)], dtype=np.uint64)
    chosen = np.zeros(n, bool)
    chosen[src] = True
    assert keys[chosen].max() < keys[~chosen].min()   # exactly the k smallest keys
    assert np.array_equal(oracle.sample_sources(n, 2, n), np.arange(n))
    assert not np.array_equal(src, oracle.sample_sources(n, 3, k))


def test_sampler_uniform_inclusion():
    n, k, seeds = 40, 10, 3000
    counts = np.zeros(n)
    for s in range(seeds):
        counts[oracle.sample_sources(n, s + 1000, k)] += 1
    p = k / n
    sd = math.sqrt(seeds * p * (1 - p))
    assert np.all(np.abs(counts - seeds * p) < 5 * sd)
    chi2 = float(np.sum((counts - seeds * p) ** 2 / (seeds * p)))
    assert chi2 < n + 6 * math.sqrt(2 * n)


def test_sampled_k_equals_n_is_exact():
    n, rp, col = oracle.generate("er", 300, 5, avg_deg=5.0)
    assert np.array_equal(oracle.betweenness_sampled(rp, col, 99, n), oracle.betweenness_exact(rp, col))


def test_sampled_estimator_is_unbiased():
    n, rp, col = oracle.generate("er", 200, 21, avg_deg=6.0)
    c = oracle.betweenness_exact(rp, col)
    runs = np.stack([oracle.betweenness_sampled(rp, col, seed, 20) for seed in range(200)])
    mean, se = runs.mean(0), runs.std(0, ddof=1) / math.sqrt(len(runs))
    mask = c > 0
    z = np.abs(mean[mask] - c[mask]) / np.maximum(se[mask], 1e-12)
    assert np.mean(z < 4) > 0.99
    assert abs(runs.sum(1).mean() - c.sum()) < 4 * runs.sum(1).std(ddof=1) / math.sqrt(len(runs))


@pytest.mark.slow
def test_sampled_top_ranks_close_to_exact():
    n, rp, col = oracle.generate("ba", 10000, 1, m0=8)
    c = oracle.betweenness_exact(rp, col)
    ch = oracle.betweenness_sampled(rp, col, 2, 256)
    top = set(np.argsort(-c)[:10].tolist())
    top_h = set(np.argsort(-ch)[:10].tolist())
    assert len(top & top_h) >= 6


# ------------------------------------------------------------------ generators (Section 5)
def check_canonical(n, rp, col):
    assert rp[0] == 0 and rp[-1] == len(col) and np.all(np.diff(rp) >= 0)
    src = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(src != col)
    key = src.astype(np.int64) * n + col
    assert np.all(np.diff(key) > 0)
    rkey = col.astype(np.int64) * n + src
    assert np.array_equal(np.sort(rkey), key)


def test_er_edge_count_and_canonical():
    n, d = 2000, 8.0
    N, p = n * (n - 1) // 2, d / (n - 1)
    ms = []
    for seed in range(1, 9):
        eu, ev = oracle.gen_er(n, d, seed)
        assert np.all(eu > ev)                       # pairs u > v, never repeated
        t = eu.astype(np.int64) * (eu - 1) // 2 + ev
        assert np.all(np.diff(t) > 0)
        ms.append(len(eu))
    sd = math.sqrt(N * p * (1 - p))
    assert all(abs(m - N * p) < 4 * sd for m in ms)
    nn, rp, col = oracle.generate("er", n, 1, avg_deg=d)
    check_canonical(nn, rp, col)
    assert len(col) == 2 * oracle.gen_er(n, d, 1)[0].size


def test_er_pair_inclusion_uniform():
    # every pair is an edge independently with probability p (tests the skip logic,
    # including the chunk boundary: n = 1500 has 1,124,250 > 2^20 pairs)
    n, p, seeds = 24, 0.3, 2500
    N = n * (n - 1) // 2
    counts = np.zeros(N)
    for s in range(seeds):
        eu, ev = oracle.gen_er(n, p * (n - 1), s + 77)
        counts[eu.astype(np.int64) * (eu - 1) // 2 + ev] += 1
    sd = math.sqrt(seeds * p * (1 - p))
    assert np.all(np.abs(counts - seeds * p) < 5 * sd)
    # chunk boundary: the density of pairs just below and above 2^20 matches p
    n2 = 1500
    p2 = 0.01
    hits = np.zeros(2)
    for s in range(40):
        eu, ev = oracle.gen_er(n2, p2 * (n2 - 1), s)
        t = eu.astype(np.int64) * (eu - 1) // 2 + ev
        hits[0] += np.sum((t >= (1 << 20) - 50000) & (t < (1 << 20)))
        hits[1] += np.sum((t >= (1 << 20)) & (t < (1 << 20) + 50000))
    for h in hits:
        assert abs(h - 40 * 50000 * p2) < 5 * math.sqrt(40 * 50000 * p2)


def test_er_complete_and_empty():
    eu, ev = oracle.gen_er(6, 5.0, 1)
    assert len(eu) == 15
    assert len(oracle.gen_er(6, 0.0, 1)[0]) == 0


def test_ba_attachment_distribution():
    # n=4, m0=1: the Batagelj-Brandes array draws r_1 in [0,2], r_2 in [0,4], r_3 in
    # [0,6]; enumerate the 105 equally likely draw sequences and compare the law of
    # the resulting edge list with the generator over many seeds.
    from collections import Counter
    law = Counter()
    for r1 in range(3):
        for r2 in range(5):
            for r3 in range(7):
                M = [0, 0]
                for e, r in ((1, r1), (2, r2), (3, r3)):
                    M.append(e)
                    M.append(M[r])
                law[tuple(M)] += 1
    seeds = 21000
    seen = Counter()
    for s in range(seeds):
        eu, ev = oracle.gen_ba(4, 1, s)
        M = []
        for a, b in zip(eu.tolist(), ev.tolist()):
            M += [a, b]
        seen[tuple(M)] += 1
    assert set(seen) <= set(law)
    chi2 = sum((seen[k] - seeds * w / 105) ** 2 / (seeds * w / 105) for k, w in law.items())
    dof = len(law) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


def test_ba_structure():
    n, m0 = 5000, 4
    eu, ev = oracle.gen_ba(n, m0, 3)
    assert len(eu) == n * m0
    assert np.array_equal(eu, np.repeat(np.arange(n), m0))
    assert np.all(ev <= eu)                              # attaches to earlier (or itself)
    nn, rp, col = oracle.generate("ba", n, 3, m0=m0)
    check_canonical(nn, rp, col)
    deg = np.diff(rp)
    assert np.all(deg[1:] >= 1) and len(col) <= 2 * n * m0
    assert deg.max() > 20 * m0                         # heavy tail: hubs exist


def test_rmat_quadrant_frequencies():
    # the benchmark's parameters, and unequal b and c so that the (0,1) and (1,0) quadrants
    # cannot be confused
    for scale, ef, a, b, c in ((12, 16, 0.57, 0.19, 0.19), (11, 16, 0.45, 0.30, 0.10)):
        eu, ev = oracle.gen_rmat(scale, ef, a, b, c, 5)
        assert len(eu) == ef << scale and eu.max() < 1 << scale and ev.max() < 1 << scale
        E = len(eu)
        for bit in (scale - 1, 0):
            ru, rv = (eu >> bit) & 1, (ev >> bit) & 1
            for (x, y), p in (((0, 0), a), ((0, 1), b), ((1, 0), c), ((1, 1), 1 - a - b - c)):
                f = np.sum((ru == x) & (rv == y))
                assert abs(f - E * p) < 5 * math.sqrt(E * p * (1 - p))
    n, rp, col = oracle.generate("rmat", 10, 1)
    check_canonical(n, rp, col)


# ------------------------------------------------------------------ closeness (Table 1)
def test_closeness_closed_forms():
    n = 9
    _, rp, col = csr(G.path(n))
    far, reach = oracle.closeness_exact(rp, col)
    i = np.arange(n)
    assert np.array_equal(far, (i * (i + 1) / 2 + (n - 1 - i) * (n - i) / 2).astype(float))
    assert np.all(reach == n - 1)
    _, rp, col = csr(G.star(7))
    far, reach = oracle.closeness_exact(rp, col)
    assert far[0] == 6 and np.all(far[1:] == 1 + 2 * 5)
    _, rp, col = csr(G.complete(6))
    far, reach = oracle.closeness_exact(rp, col)
    assert np.all(far == 5) and np.all(reach == 5)
    r = 6
    _, rp, col = csr(G.cycle(2 * r + 1))
    far, _ = oracle.closeness_exact(rp, col)
    assert np.all(far == r * (r + 1))


@pytest.mark.parametrize("graph", [G.gnp(40, 0.08, 3), G.grid(5, 7), G.random_tree(50, 2),
                                   G.disjoint_union(G.path(6), G.gnp(20, 0.2, 4), G.complete(1))])
def test_closeness_matches_floyd_warshall(graph):
    n, rp, col = csr(graph)
    d = floyd_warshall(*graph)
    far, reach = oracle.closeness_exact(rp, col)
    dd = np.where(d > 0, d, 0)
    assert np.array_equal(far, dd.sum(0).astype(float))
    assert np.array_equal(reach, (d > 0).sum(0).astype(float))


def test_closeness_sampled_unbiased_and_k_equals_n():
    n, rp, col = oracle.generate("er", 150, 7, avg_deg=5.0)
    far, reach = oracle.closeness_exact(rp, col)
    fs, rs = oracle.closeness_sampled(rp, col, 3, n)
    assert np.array_equal(fs, far) and np.array_equal(rs, reach)
    runs = np.stack([oracle.closeness_sampled(rp, col, s, 15)[0] for s in range(300)])
    mean, se = runs.mean(0), runs.std(0, ddof=1) / np.sqrt(len(runs))
    z = np.abs(mean - far) / np.maximum(se, 1e-12)
    assert np.mean(z < 4) > 0.99


# ------------------------------------------------------------------ edge betweenness (Section 4.3)
def edge_values(n, rp, col, e):
    """{(a, b), a < b: value} from per-arc scores; both arcs of an edge must agree."""
    out = {}
    for a in range(n):
        for j in range(rp[a], rp[a + 1]):
            b = int(col[j])
            key = (min(a, b), max(a, b))
            if key in out:
                assert out[key] == e[j], key
            out[key] = e[j]
    return out


def test_edge_betweenness_closed_forms():
    n = 10
    _, rp, col = csr(G.path(n))
    ev = edge_values(n, rp, col, oracle.edge_betweenness_exact(rp, col))
    assert all(ev[(i, i + 1)] == (i + 1) * (n - 1 - i) for i in range(n - 1))
    _, rp, col = csr(G.star(8))
    assert np.all(oracle.edge_betweenness_exact(rp, col) == 7)
    _, rp, col = csr(G.complete(7))
    assert np.all(oracle.edge_betweenness_exact(rp, col) == 1)
    r = 5
    _, rp, col = csr(G.cycle(2 * r + 1))
    assert np.allclose(oracle.edge_betweenness_exact(rp, col), r * (r + 1) / 2, rtol=1e-14)
    _, rp, col = csr(G.cycle(2 * r))
    assert np.allclose(oracle.edge_betweenness_exact(rp, col), r * r / 2, rtol=1e-14)
    a, b = 4, 7
    _, rp, col = csr(G.complete_bipartite(a, b))
    assert np.allclose(oracle.edge_betweenness_exact(rp, col), 1 + (a - 1) / b + (b - 1) / a, rtol=1e-14)


@pytest.mark.parametrize("seed", [1, 2])
def test_edge_betweenness_tree_side_products(seed):
    n = 200
    g = G.random_tree(n, seed)
    _, rp, col = csr(g)
    ev = edge_values(n, rp, col, oracle.edge_betweenness_exact(rp, col))
    adj = [[] for _ in range(n)]
    for x, y in zip(g[1].tolist(), g[2].tolist()):
        adj[x].append(y)
        adj[y].append(x)
    for (x, y), val in list(ev.items())[::5]:
        seen, stack = {x, y}, [y]          # the side of y once {x, y} is cut
        while stack:
            z = stack.pop()
            for w in adj[z]:
                if w not in seen:
                    seen.add(w)
                    stack.append(w)
        side = len(seen) - 1
        assert val == side * (n - side)


def _edge_close(n, rp, col, e, ref):
    ev = edge_values(n, rp, col, e)
    assert set(ev) == set(ref)
    return all(math.isclose(ev[key], float(ref[key]), rel_tol=1e-12, abs_tol=1e-12) for key in ref)


def test_edge_betweenness_all_graphs_on_5_vertices():
    from bruteforce import edge_betweenness_bruteforce
    for mask in range(0, 1 << 10, 3):
        g = G.from_mask(5, mask)
        n, rp, col = csr(g)
        assert _edge_close(n, rp, col, oracle.edge_betweenness_exact(rp, col), edge_betweenness_bruteforce(*g)), mask


@pytest.mark.parametrize("seed", range(12))
def test_edge_betweenness_random_small_bruteforce(seed):
    from bruteforce import edge_betweenness_bruteforce
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(6, 12))
    g = (G.gnp(n, float(rng.uniform(0.2, 0.6)), seed) if seed % 3 else
         G.disjoint_union(G.gnp(n // 2, 0.6, seed), G.random_tree(n - n // 2, seed)))
    n, rp, col = csr(g)
    assert _edge_close(n, rp, col, oracle.edge_betweenness_exact(rp, col), edge_betweenness_bruteforce(*g))


@pytest.mark.parametrize("graph", [G.gnp(120, 0.05, 4), G.grid(9, 13),
                                   G.disjoint_union(G.cycle(30), G.gnp(60, 0.1, 5), G.star(9))])
def test_edge_betweenness_invariants(graph):
    # sum over edges = sum over reachable unordered pairs of d(s, t); and at every vertex the
    # incident edges carry 2 c_B(v) + reach(v) (an interior vertex of a path meets two of
    # its edges, an endpoint one)
    n, rp, col = csr(graph)
    e = oracle.edge_betweenness_exact(rp, col)
    d = floyd_warshall(*graph)
    assert math.isclose(e.sum() / 2, d[d > 0].sum() / 2, rel_tol=1e-12)
    cb = oracle.betweenness_exact(rp, col)
    _, reach = oracle.closeness_exact(rp, col)
    inc = np.array([e[rp[v]:rp[v + 1]].sum() for v in range(n)])
    assert np.allclose(inc, 2 * cb + reach, rtol=1e-12, atol=1e-12)


def test_edge_betweenness_sampled_unbiased_and_k_equals_n():
    n, rp, col = oracle.generate("er", 120, 5, avg_deg=5.0)
    e = oracle.edge_betweenness_exact(rp, col)
    assert np.array_equal(oracle.edge_betweenness_sampled(rp, col, 4, n), e)
    runs = np.stack([oracle.edge_betweenness_sampled(rp, col, s, 12) for s in range(300)])
    mean, se = runs.mean(0), runs.std(0, ddof=1) / np.sqrt(len(runs))
    z = np.abs(mean - e) / np.maximum(se, 1e-12)
    assert np.mean(z < 4) > 0.99


# ------------------------------------------------------------------ error-bounded estimate (Section 3.2)
def test_vertex_diameter_estimate_closed_forms():
    for n in (1, 2, 7, 30):
        _, rp, col = csr(G.path(n))
        assert oracle.vertex_diameter_estimate(rp, col) == n      # 2(n-1)+1 capped by |C| = n
    _, rp, col = csr(G.star(9))
    assert oracle.vertex_diameter_estimate(rp, col) == 3          # from the centre: ecc 1
    _, rp, col = csr(G.cycle(11))
    assert oracle.vertex_diameter_estimate(rp, col) == 11         # ecc 5 -> 11 = |C|
    _, rp, col = csr(G.grid(4, 6))
    assert oracle.vertex_diameter_estimate(rp, col) == 17         # corner ecc 8 -> 17 <= 24
    _, rp, col = csr(G.disjoint_union(G.star(5), G.path(9), G.complete(1)))
    assert oracle.vertex_diameter_estimate(rp, col) == 9          # the largest component bound


@pytest.mark.parametrize("seed", range(6))
def test_vertex_diameter_estimate_bounds(seed):
    g = G.gnp(40, 0.06 + 0.02 * seed, seed) if seed % 2 else G.random_tree(40, seed)
    n, rp, col = csr(g)
    d = floyd_warshall(*g)
    vd_true = int(d.max()) + 1                                   # vertices on a longest shortest path
    vd = oracle.vertex_diameter_estimate(rp, col)
    assert vd_true <= vd <= 2 * vd_true + 1


def test_rk_sample_count_hand_values():
    # r = ceil(0.5 / eps^2 * (floor(log2(max(VD - 2, 1))) + 1 + ln(1 / delta))), worked by hand
    assert oracle.rk_sample_count(0.1, 0.1, 10) == 316     # 50 * (3 + 1 + 2.302585) = 315.13
    assert oracle.rk_sample_count(0.1, 0.1, 12) == 316     # floor(log2 10) = 3 as well
    assert oracle.rk_sample_count(0.1, 0.1, 11) == 316
    assert oracle.rk_sample_count(0.1, 0.1, 18) == 366     # 50 * (4 + 1 + 2.302585) = 365.13
    assert oracle.rk_sample_count(0.05, 0.01, 3) == 1122   # 200 * (0 + 1 + 4.605170) = 1121.03
    assert oracle.rk_sample_count(0.2, 0.5, 2) == 22       # 12.5 * (1 + 0.693147) = 21.16
    with pytest.raises(oracle.OracleError):
        oracle.rk_sample_count(0.0, 0.1, 5)
    with pytest.raises(oracle.OracleError):
        oracle.rk_sample_count(0.1, 1.0, 5)


def test_rk_pair_and_path_laws():
    # 3 x 3 grid: 72 ordered pairs equally likely; between opposite corners the 6 shortest
    # paths equally likely
    n, rp, col = csr(G.grid(3, 3))
    N = 20000
    pairs, paths = {}, {}
    for i in range(N):
        u, v, p = oracle.rk_path(rp, col, 11, i)
        assert u != v
        pairs[(u, v)] = pairs.get((u, v), 0) + 1
        if (u, v) == (0, 8):
            paths[tuple(p)] = paths.get(tuple(p), 0) + 1
    assert len(pairs) == 72
    e = N / 72
    chi2 = sum((c - e) ** 2 / e for c in pairs.values())
    assert chi2 < 71 + 5 * math.sqrt(2 * 71)
    assert len(paths) == 6
    tot = sum(paths.values())
    chi2 = sum((c - tot / 6) ** 2 / (tot / 6) for c in paths.values())
    assert chi2 < 5 + 5 * math.sqrt(10)


def test_rk_tree_paths_are_the_tree_paths():
    n = 60
    g = G.random_tree(n, 4)
    _, rp, col = csr(g)
    for i in range(200):
        u, v, p = oracle.rk_path(rp, col, 2, i)
        dist, _ = oracle.bfs(rp, col, u)
        # walk back from v by decreasing distance: unique in a tree
        w, want = v, []
        while dist[w] > 1:
            w = next(int(c) for c in col[rp[w]:rp[w + 1]] if dist[c] == dist[w] - 1)
            want.append(w)
        assert p.tolist() == want


def test_rk_unbiased_and_within_epsilon():
    n, rp, col = oracle.generate("er", 80, 3, avg_deg=4.0)
    exact = oracle.betweenness_exact(rp, col)
    eps, delta = 0.05, 0.1
    runs, misses = [], 0
    for s in range(60):
        sc, r, vd = oracle.betweenness_rk(rp, col, eps, delta, s)
        runs.append(sc)
        misses += np.max(np.abs(sc - exact)) * 2 / (n * (n - 1)) > eps
    assert misses <= 6 + 3                                      # P(miss) <= delta = 0.1
    runs = np.stack(runs)
    mean, se = runs.mean(0), runs.std(0, ddof=1) / np.sqrt(len(runs))
    z = np.abs(mean - exact) / np.maximum(se, 1e-12)
    assert np.mean(z < 4) > 0.97


def test_rk_small_vertex_diameter_gives_zero():
    # complete graph: no shortest path has an interior vertex
    _, rp, col = csr(G.complete(6))
    sc, r, vd = oracle.betweenness_rk(rp, col, 0.2, 0.2, 1)
    assert vd == 3 and r == oracle.rk_sample_count(0.2, 0.2, 3) and np.all(sc == 0)


# ------------------------------------------------------------------ weighted graphs (Sections 2.3, 3.4)
def test_edge_weights_symmetric_and_in_range():
    n, rp, col = oracle.generate("er", 300, 2, avg_deg=6.0)
    w = oracle.edge_weights(rp, col, 9, 7)
    assert w.min() >= 1 and w.max() <= 7 and len(set(w.tolist())) == 7
    for u in range(0, n, 7):
        for j in range(rp[u], rp[u + 1]):
            v = col[j]
            r = rp[v] + int(np.searchsorted(col[rp[v]:rp[v + 1]], u))
            assert w[r] == w[j]
    assert np.all(oracle.edge_weights(rp, col, 9, 1) == 1)


@pytest.mark.parametrize("graph", [G.grid(6, 7), G.gnp(150, 0.04, 2), G.hypercube(5),
                                   G.disjoint_union(G.cycle(12), G.star(6), G.complete(1))])
def test_weighted_reduces_to_unweighted(graph):
    n, rp, col = csr(graph)
    base = oracle.betweenness_exact(rp, col)
    for c in (1, 3):
        w = np.full(len(col), c, np.int32)
        assert np.allclose(oracle.betweenness_weighted_exact(rp, col, w), base, rtol=1e-12, atol=1e-12)
        for s in (0, n // 2):
            d, sg = oracle.sssp_weighted(rp, col, w, s)
            d0, s0 = oracle.bfs(rp, col, s)
            assert np.array_equal(d, np.where(d0 >= 0, c * d0.astype(np.int64), -1))
            assert np.array_equal(sg, s0)


def test_weighted_trees_and_paths_ignore_weights():
    for g in (G.path(20), G.random_tree(120, 6)):
        n, rp, col = csr(g)
        w = oracle.edge_weights(rp, col, 4, 9)
        assert np.allclose(oracle.betweenness_weighted_exact(rp, col, w), oracle.betweenness_exact(rp, col),
                           rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(10))
def test_weighted_bruteforce_small(seed):
    from bruteforce import weighted_bruteforce
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(5, 9))
    g = G.gnp(n, float(rng.uniform(0.3, 0.7)), seed) if seed % 3 else G.disjoint_union(G.cycle(4), G.gnp(n - 4, 0.6, seed))
    n, rp, col = csr(g)
    w = oracle.edge_weights(rp, col, seed, 1 + seed % 4)   # wmax 1..4: many equal-length ties
    dist, sigma, c = weighted_bruteforce(rp, col, w)
    for s in range(n):
        d, sg = oracle.sssp_weighted(rp, col, w, s)
        assert d.tolist() == dist[s]
        assert sg.tolist() == [sigma[s][t] if dist[s][t] >= 0 else 0 for t in range(n)]
    got = oracle.betweenness_weighted_exact(rp, col, w)
    assert np.allclose(got, [float(x) for x in c], rtol=1e-12, atol=1e-12)


def test_weighted_cycle_with_a_heavy_edge():
    # C_4 = 0-1-2-3-0 with w(3,0) = 3: 0 reaches 3 by 0-1-2-3 (length 3) and by the edge
    # (length 3), so the pair {0, 3} splits over two paths; every other pair has one path
    n, u, v = G.cycle(4)
    rp, col = oracle.csr_build(n, u, v)
    w = np.ones(len(col), np.int32)
    for j in range(len(col)):
        a = int(np.searchsorted(rp, j, side="right") - 1)
        if {a, int(col[j])} == {0, 3}:
            w[j] = 3
    d, sg = oracle.sssp_weighted(rp, col, w, 0)
    assert d.tolist() == [0, 1, 2, 3] and sg.tolist() == [1, 1, 1, 2]
    c = oracle.betweenness_weighted_exact(rp, col, w)
    # vertex 1: {0,2} (1 path, via 1) + {0,3} (1 of 2) = 1.5; vertex 2: {1,3} + {0,3}/2 = 1.5;
    # vertex 0: {1,3}? 1-0-3 weighs 4 > 1-2-3: 0; vertex 3: {0,2}? 0-3-2 weighs 4: 0
    assert np.allclose(c, [0.0, 1.5, 1.5, 0.0], rtol=1e-14)


def test_weighted_sampled_k_equals_n():
    n, rp, col = oracle.generate("ba", 400, 3, m0=3)
    w = oracle.edge_weights(rp, col, 5, 10)
    assert np.array_equal(oracle.betweenness_weighted_sampled(rp, col, w, 8, n),
                          oracle.betweenness_weighted_exact(rp, col, w))


def test_rk_counts_in_ranges_add_up_to_the_estimate():
    n, rp, col = oracle.generate("er", 300, 6, avg_deg=5.0)
    sc, r, vd = oracle.betweenness_rk(rp, col, 0.1, 0.1, 4)
    cuts = [0, 7, 100, r // 2, r]
    counts = sum(oracle.rk_counts(rp, col, 4, a, b) for a, b in zip(cuts[:-1], cuts[1:]))
    assert np.array_equal(counts.astype(np.float64) * (n * (n - 1) / (2.0 * r)), sc)


def test_edge_betweenness_single_source_bruteforce():
    # one source s: the edge {u, v} scores sum_t sigma_st({u, v}) / sigma_st on both of its arcs
    # (a sum over one source is not symmetric in the edge's direction, unlike a sum over all)
    from bruteforce import adjacency, enumerate_shortest_paths
    for g in (G.gnp(9, 0.4, 3), G.grid(3, 4), G.disjoint_union(G.cycle(6), G.star(4))):
        n, rp, col = csr(g)
        adj = adjacency(*g)
        for s in range(n):
            ref = {}
            for t in range(n):
                if t == s:
                    continue
                ps = enumerate_shortest_paths(adj, s, t)
                for p in ps:
                    for x, y in zip(p[:-1], p[1:]):
                        key = (min(x, y), max(x, y))
                        ref[key] = ref.get(key, Fraction(0)) + Fraction(1, len(ps))
            e = oracle.edge_betweenness_sources(rp, col, np.array([s], np.int32), 1.0)
            ev = edge_values(n, rp, col, e)
            for key, val in ev.items():
                assert math.isclose(val, float(ref.get(key, 0)), rel_tol=1e-12, abs_tol=1e-12), (s, key)
