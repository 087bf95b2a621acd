"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Every function returns ``(n, u, v)``: a vertex count and two int32 arrays of edge end
points (an undirected edge list, possibly with self-loops or duplicates where a test
wants them).  Nothing here computes distances, path counts or dependencies; turning an
edge list into a canonical CSR is each side's own job.
"""
from __future__ import annotations

import itertools

import numpy as np


def _edges(n, pairs):
    pairs = list(pairs)
    if not pairs:
        return n, np.zeros(0, np.int32), np.zeros(0, np.int32)
    a = np.asarray(pairs, dtype=np.int64)
    return n, a[:, 0].astype(np.int32), a[:, 1].astype(np.int32)


def path(n):
    return _edges(n, ((i, i + 1) for i in range(n - 1)))


def cycle(n):
    return _edges(n, ((i, (i + 1) % n) for i in range(n)))


def star(n):
    """Centre 0, leaves 1..n-1."""
    return _edges(n, ((0, i) for i in range(1, n)))


def complete(n):
    return _edges(n, itertools.combinations(range(n), 2))


def complete_bipartite(a, b):
    """Side A = 0..a-1, side B = a..a+b-1."""
    return _edges(a + b, ((i, a + j) for i in range(a) for j in range(b)))


def grid(rows, cols):
    """Vertex (i, j) has id i*cols + j."""
    pairs = []
    for i in range(rows):
        for j in range(cols):
            if j + 1 < cols:
                pairs.append((i * cols + j, i * cols + j + 1))
            if i + 1 < rows:
                pairs.append((i * cols + j, (i + 1) * cols + j))
    return _edges(rows * cols, pairs)


def hypercube(d):
    n = 1 << d
    return _edges(n, ((x, x ^ (1 << b)) for x in range(n) for b in range(d) if x < x ^ (1 << b)))


def hypercube_edges(d):
    """Edge list (u < v) of the hypercube Q_d built with numpy (for large d)."""
    n = 1 << d
    x = np.repeat(np.arange(n, dtype=np.int64), d)
    y = x ^ (1 << np.tile(np.arange(d, dtype=np.int64), n))
    keep = x < y
    return n, x[keep].astype(np.int32), y[keep].astype(np.int32)


def random_tree(n, seed):
    """Vertex i > 0 hangs off a uniformly chosen earlier vertex; ids are then permuted."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    pairs = [(perm[i], perm[int(rng.integers(0, i))]) for i in range(1, n)]
    return _edges(n, pairs)


def gnp(n, p, seed):
    """Dense-sampled G(n, p) for small n (numpy generator, not the library's ER)."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    return n, iu[keep].astype(np.int32), ju[keep].astype(np.int32)


def from_mask(n, mask):
    """The labelled graph on n vertices whose edge set is the bit mask over the
    pairs of itertools.combinations(range(n), 2)."""
    pairs = [pq for b, pq in enumerate(itertools.combinations(range(n), 2)) if mask >> b & 1]
    return _edges(n, pairs)


def disjoint_union(*graphs):
    n0, us, vs = 0, [], []
    for n, u, v in graphs:
        us.append(u + n0)
        vs.append(v + n0)
        n0 += n
    return n0, np.concatenate(us).astype(np.int32), np.concatenate(vs).astype(np.int32)


def noisy(graph, seed, dup_frac=0.3, loops=3):
    """The same simple graph written with duplicates, reversed copies, self-loops and a
    shuffled order: what a canonicalising CSR builder must reduce to the simple graph."""
    n, u, v = graph
    rng = np.random.default_rng(seed)
    m = len(u)
    k = int(dup_frac * m)
    idx = rng.integers(0, max(m, 1), k) if m else np.zeros(0, np.int64)
    uu = np.concatenate([u, v[idx], rng.integers(0, n, loops)])
    vv = np.concatenate([v, u[idx], np.zeros(loops, np.int64)])
    vv[len(u) + k:] = uu[len(u) + k:]
    order = rng.permutation(len(uu))
    return n, uu[order].astype(np.int32), vv[order].astype(np.int32)


def relabel(graph, seed):
    n, u, v = graph
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    return n, perm[u], perm[v]


def with_hubs(graph, degrees, seed):
    """The graph plus one hub per entry of `degrees`: hub i (vertex i) gets edges to
    degrees[i] distinct other vertices chosen at random (so rows cross the 256-arc chunk
    boundary of the GPU kernels when asked to)."""
    n, u, v = graph
    rng = np.random.default_rng(seed)
    us, vs = [u], [v]
    for h, d in enumerate(degrees):
        others = rng.choice(np.setdiff1d(np.arange(n), [h]), size=d, replace=False)
        us.append(np.full(d, h, np.int64))
        vs.append(others)
    return n, np.concatenate(us).astype(np.int32), np.concatenate(vs).astype(np.int32)
