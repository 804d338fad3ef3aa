"""Seeded synthetic inputs (graphs, vertex weights, start colourings).

The paper evaluates on DIMACS/COLOR benchmark files, which this project does not ship; seeded
synthetic graphs of the same kinds stand in for them: uniform random graphs G(n, p) (the DSJCn.d
family is G(n, p) with p = d/10), planted k-partite graphs (a hidden k-colouring with edges only
across parts, like the flat_n_k family) and vertex weights uniform in 1..100 for the weighted
problem. This module holds none of the method's arithmetic: it only produces inputs, from
numpy's PCG64 generator, and both the CUDA path and the oracle consume what it returns.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), 0x2109_05948 & 0xFFFFFFFF]))


def edges_to_adj(n: int, edges: np.ndarray) -> np.ndarray:
    """Dense symmetric 0/1 adjacency (uint8, n x n) of an undirected edge list."""
    adj = np.zeros((n, n), np.uint8)
    if len(edges):
        adj[edges[:, 0], edges[:, 1]] = 1
        adj[edges[:, 1], edges[:, 0]] = 1
    return adj


def adj_to_edges(adj: np.ndarray) -> np.ndarray:
    u, v = np.nonzero(np.triu(adj, 1))
    return np.stack([u, v], 1).astype(np.int32)


def gnp(n: int, p: float, seed: int) -> np.ndarray:
    """Edge list (m x 2 int32, u < v) of a uniform random graph G(n, p)."""
    r = _rng(seed).random((n, n))
    iu = np.triu_indices(n, 1)
    keep = r[iu] < p
    return np.stack([iu[0][keep], iu[1][keep]], 1).astype(np.int32)


def planted(n: int, k: int, p: float, seed: int):
    """A graph with a hidden k-colouring: vertices are shuffled and dealt into k parts of sizes
    floor(n/k) or ceil(n/k); each pair of vertices in different parts is an edge with
    probability p. Returns (edges, part) with part[v] the hidden colour of v."""
    g = _rng(seed)
    perm = g.permutation(n)
    part = np.empty(n, np.int32)
    part[perm] = np.arange(n) % k
    r = g.random((n, n))
    iu = np.triu_indices(n, 1)
    keep = (r[iu] < p) & (part[iu[0]] != part[iu[1]])
    return np.stack([iu[0][keep], iu[1][keep]], 1).astype(np.int32), part


def weights(n: int, seed: int, lo: int = 1, hi: int = 100) -> np.ndarray:
    """Integer vertex weights uniform in lo..hi (int32)."""
    return _rng(seed + 0x5EED).integers(lo, hi + 1, size=n).astype(np.int32)


def random_colorings(pop: int, n: int, k: int, seed: int) -> np.ndarray:
    """Uniform start colourings (pop x n int16) drawn by numpy, for tests that feed both sides."""
    return _rng(seed + 0xC0105).integers(0, k, size=(pop, n)).astype(np.int16)


def complete(n: int) -> np.ndarray:
    iu = np.triu_indices(n, 1)
    return np.stack(iu, 1).astype(np.int32)


def cycle(n: int) -> np.ndarray:
    return np.array([[i, (i + 1) % n] if i < (i + 1) % n else [(i + 1) % n, i] for i in range(n)], np.int32)


def random_bipartite(n: int, p: float, seed: int) -> np.ndarray:
    e, _ = planted(n, 2, p, seed)
    return e


def uneven_batch(num_graphs: int = 64, seed: int = 0, n_lo: int = 100, n_hi: int = 1000):
    """The uneven multi-graph workload: num_graphs graphs with n uniform in [n_lo, n_hi], density
    cycling through {0.1, 0.5, 0.9}, every odd-indexed graph planted, k = n // 10 colours.
    Returns a list of dicts (n, k, p, planted, edges)."""
    g = _rng(seed + 0xBA7C)
    out = []
    for i in range(num_graphs):
        n = int(g.integers(n_lo, n_hi + 1))
        p = (0.1, 0.5, 0.9)[i % 3]
        k = max(2, n // 10)
        if i % 2 == 1:
            e, _ = planted(n, k, p, seed * 1000 + i)
        else:
            e = gnp(n, p, seed * 1000 + i)
        out.append(dict(n=n, k=k, p=p, planted=bool(i % 2), edges=e))
    return out
