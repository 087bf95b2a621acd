"""Independent brute-force references for tiny graphs (tests only).

None of these use BFS or Brandes' recurrences:
  * ``floyd_warshall`` - all-pairs hop distances by the Floyd-Warshall relaxation;
  * ``enumerate_shortest_paths`` - for each pair, simple paths of length 1, 2, ... are
    enumerated by depth-limited DFS until the first length that has any; those paths are
    the shortest ones, so sigma_st and sigma_st(v) are plain counts;
  * ``betweenness_bruteforce`` - c(v) = sum over unordered pairs {s,t}, s != v != t, of
    sigma_st(v)/sigma_st, straight from the definition.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def adjacency(n, u, v):
    adj = [set() for _ in range(n)]
    for a, b in zip(np.asarray(u).tolist(), np.asarray(v).tolist()):
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    return adj


def floyd_warshall(n, u, v):
    INF = np.iinfo(np.int64).max // 4
    d = np.full((n, n), INF, dtype=np.int64)
    np.fill_diagonal(d, 0)
    for a, b in zip(np.asarray(u).tolist(), np.asarray(v).tolist()):
        if a != b:
            d[a, b] = d[b, a] = 1
    for k in range(n):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    d[d >= INF] = -1
    return d


def _paths_of_length(adj, s, t, L):
    out, stack = [], [s]
    on = {s}

    def dfs(x, left):
        if left == 0:
            if x == t:
                out.append(tuple(stack))
            return
        for y in adj[x]:
            if y in on:
                continue
            if left == 1 and y != t:
                continue
            on.add(y)
            stack.append(y)
            dfs(y, left - 1)
            stack.pop()
            on.discard(y)

    dfs(s, L)
    return out


def enumerate_shortest_paths(adj, s, t):
    """All shortest s-t paths (as vertex tuples); [] if t is unreachable."""
    n = len(adj)
    if s == t:
        return [(s,)]
    for L in range(1, n):
        ps = _paths_of_length(adj, s, t, L)
        if ps:
            return ps
    return []


def sssp_bruteforce(n, u, v, s):
    adj = adjacency(n, u, v)
    dist = np.full(n, -1, np.int64)
    sigma = np.zeros(n, dtype=object)
    for t in range(n):
        ps = enumerate_shortest_paths(adj, s, t)
        if ps:
            dist[t] = len(ps[0]) - 1
            sigma[t] = len(ps)
    return dist, sigma


def betweenness_bruteforce(n, u, v):
    """Exact rationals, unordered pairs, endpoints excluded, unreachable pairs add 0."""
    adj = adjacency(n, u, v)
    c = [Fraction(0)] * n
    for s, t in itertools.combinations(range(n), 2):
        ps = enumerate_shortest_paths(adj, s, t)
        if not ps:
            continue
        cnt = [0] * n
        for p in ps:
            for x in p[1:-1]:
                cnt[x] += 1
        for x in range(n):
            if cnt[x]:
                c[x] += Fraction(cnt[x], len(ps))
    return c


def edge_betweenness_bruteforce(n, u, v):
    """{(a, b), a < b: exact rational edge betweenness}: over unordered reachable pairs
    {s, t}, the fraction of shortest s-t paths that use the edge."""
    adj = adjacency(n, u, v)
    c = {}
    for a in range(n):
        for b in adj[a]:
            if a < b:
                c[(a, b)] = Fraction(0)
    for s, t in itertools.combinations(range(n), 2):
        ps = enumerate_shortest_paths(adj, s, t)
        if not ps:
            continue
        for p in ps:
            for x, y in zip(p[:-1], p[1:]):
                c[(min(x, y), max(x, y))] += Fraction(1, len(ps))
    return c


def weighted_bruteforce(rp, col, w):
    """(dist, sigma, c): by enumerating every simple path of a small weighted graph (no
    Dijkstra): dist[s][t] = least total weight (-1 unreachable), sigma[s][t] = number of
    simple paths of that weight, c[v] = exact rational betweenness (unordered pairs)."""
    rp, col, w = list(map(int, rp)), list(map(int, col)), list(map(int, w))
    n = len(rp) - 1
    best = [[None] * n for _ in range(n)]
    paths = [[[] for _ in range(n)] for _ in range(n)]

    def dfs(s, v, seen, path, length):
        if best[s][v] is None or length < best[s][v]:
            best[s][v] = length
            paths[s][v] = [tuple(path)]
        elif length == best[s][v]:
            paths[s][v].append(tuple(path))
        for j in range(rp[v], rp[v + 1]):
            x = col[j]
            if x not in seen:
                seen.add(x)
                path.append(x)
                dfs(s, x, seen, path, length + w[j])
                path.pop()
                seen.remove(x)

    for s in range(n):
        dfs(s, s, {s}, [s], 0)
    dist = [[-1 if best[s][t] is None else best[s][t] for t in range(n)] for s in range(n)]
    sigma = [[len(paths[s][t]) for t in range(n)] for s in range(n)]
    c = [Fraction(0)] * n
    for s, t in itertools.combinations(range(n), 2):
        ps = paths[s][t]
        if not ps:
            continue
        for p in ps:
            for x in p[1:-1]:
                c[x] += Fraction(1, len(ps))
    return dist, sigma, c
