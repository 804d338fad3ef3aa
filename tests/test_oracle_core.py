"""Pins of the oracle's RNG, initialisation, conflict table and TabuCol against facts fixed by
the paper's definitions and by mathematics (CPU only)."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2109_05948_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------------------------------------
# Philox4x32-10
# ------------------------------------------------------------------------------------------------
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = [int(x, 16) for x in line.split()]
                rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox(ctr, key)) == expect


def test_draw_is_philox_with_seed_key():
    seed = 0x1234_5678_9ABC_DEF0
    got = oracle.draw(seed, 7, 8, 9, oracle.TAG_TABU)
    ref = oracle.philox([7, 8, 9, oracle.TAG_TABU], [seed & 0xFFFFFFFF, seed >> 32])
    assert list(got) == list(ref)


def test_init_colors_uniform_and_in_range():
    n, k, pop = 500, 48, 64
    col = oracle.init_colors(n, k, pop, seed=0)
    assert col.min() >= 0 and col.max() < k
    counts = np.bincount(col.ravel(), minlength=k)
    expected = n * pop / k
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 100.0  # k-1 = 47 degrees of freedom; p(chi2 > 100) < 1e-5
    # each entry is the high word of r0 * k for counter (v, 0, individual, INIT)
    r = oracle.draw(0, 3, 0, 5, oracle.TAG_INIT)
    assert col[5, 3] == (int(r[0]) * k) >> 32
    # a different individual base shifts the streams
    col2 = oracle.init_colors(n, k, 2, seed=0, ind_base=5)
    assert np.array_equal(col2[0], col[5])


# ------------------------------------------------------------------------------------------------
# conflict table and objective (Eq. f)
# ------------------------------------------------------------------------------------------------
def _f_from_edges(edges, col):
    return int(np.sum(col[edges[:, 0]] == col[edges[:, 1]]))


def test_gamma_and_f_recount():
    n, k = 80, 6
    e = inputs.gnp(n, 0.3, seed=4)
    adj = inputs.edges_to_adj(n, e)
    col = inputs.random_colorings(1, n, k, seed=1)[0]
    g, f = oracle.gamma(adj, k, col)
    assert f == _f_from_edges(e, col)
    ref = np.zeros((n, k), np.int64)
    np.add.at(ref, (e[:, 0], col[e[:, 1]]), 1)
    np.add.at(ref, (e[:, 1], col[e[:, 0]]), 1)
    assert np.array_equal(g, ref)


def test_graph_csr_matches_adjacency():
    n = 70
    e = inputs.gnp(n, 0.4, seed=2)
    adj = inputs.edges_to_adj(n, e)
    off, idx, bits = oracle.graph_csr(adj)
    for v in range(n):
        assert list(idx[off[v]:off[v + 1]]) == list(np.nonzero(adj[v])[0])
        row = np.unpackbits(bits[v].view(np.uint8), bitorder="little")[:n]
        assert np.array_equal(row, adj[v])


# ------------------------------------------------------------------------------------------------
# TabuCol pins
# ------------------------------------------------------------------------------------------------
def _min_conflicts_brute(n, edges, k):
    """Exact minimum number of conflicting edges over all k-colourings (tiny n)."""
    best = None
    cols = np.array(list(itertools.product(range(k), repeat=n)), np.int16)
    same = cols[:, edges[:, 0]] == cols[:, edges[:, 1]]
    best = int(same.sum(1).min())
    return best


def _chromatic_brute(n, edges):
    for k in range(1, n + 1):
        if _min_conflicts_brute(n, edges, k) == 0:
            return k
    return n


def _run(adj, k, seed, iters=10_000, ind=0, check=False):
    n = adj.shape[0]
    start = oracle.init_colors(n, k, 1, seed, ind_base=ind)[0]
    return oracle.tabucol(adj, k, start, iters, seed=seed, ind=ind, check=check)


@pytest.mark.parametrize("gseed", [1, 2, 3, 4, 5])
def test_tabucol_brute_force_chromatic(gseed):
    n = 9
    e = inputs.gnp(n, 0.5, seed=gseed)
    adj = inputs.edges_to_adj(n, e)
    chi = _chromatic_brute(n, e)
    # k = chi: a legal colouring exists and the search finds it
    r = _run(adj, chi, seed=gseed, check=True)
    assert r["best_f"] == 0 and _f_from_edges(e, r["best_col"]) == 0
    if chi >= 2:
        # k = chi - 1: no legal colouring; best_f never drops below the exact minimum and reaches it
        mc = _min_conflicts_brute(n, e, chi - 1)
        assert mc >= 1
        r = _run(adj, chi - 1, seed=gseed, iters=3000, check=True)
        assert r["best_f"] == mc == _f_from_edges(e, r["best_col"])
        assert r["iters"] == 3000


@pytest.mark.parametrize("n,k", [(8, 3), (10, 4), (12, 5)])
def test_tabucol_complete_graph_closed_form(n, k):
    adj = inputs.edges_to_adj(n, inputs.complete(n))
    sizes = [n // k + (1 if c < n % k else 0) for c in range(k)]
    closed = sum(s * (s - 1) // 2 for s in sizes)
    r = _run(adj, k, seed=11, iters=2000, check=True)
    assert r["best_f"] == closed


@pytest.mark.parametrize("n", [5, 9, 31])
def test_tabucol_odd_cycle_two_colours(n):
    e = inputs.cycle(n)
    adj = inputs.edges_to_adj(n, e)
    r = _run(adj, 2, seed=3, iters=2000, check=True)
    assert r["best_f"] == 1 == _f_from_edges(e, r["best_col"])


@pytest.mark.parametrize("n", [6, 10, 40])
def test_tabucol_even_cycle_and_bipartite(n):
    adj = inputs.edges_to_adj(n, inputs.cycle(n))
    assert _run(adj, 2, seed=5, check=True)["best_f"] == 0
    e = inputs.random_bipartite(n, 0.4, seed=n)
    adj = inputs.edges_to_adj(n, e)
    r = _run(adj, 2, seed=6, check=True)
    assert r["best_f"] == 0 and _f_from_edges(e, r["best_col"]) == 0


def test_tabucol_planted_reaches_zero():
    n, k = 120, 6
    e, part = inputs.planted(n, k, 0.5, seed=9)
    adj = inputs.edges_to_adj(n, e)
    assert _f_from_edges(e, part) == 0
    r = _run(adj, k, seed=9, iters=20_000, check=True)
    assert r["best_f"] == 0 and _f_from_edges(e, r["best_col"]) == 0
    assert r["iters"] < 20_000  # stopped at f = 0


def test_tabucol_trace_moves_are_minimal_conflicting_moves():
    n, k = 40, 4
    e = inputs.gnp(n, 0.3, seed=8)
    adj = inputs.edges_to_adj(n, e)
    start = inputs.random_colorings(1, n, k, seed=8)[0]
    r = oracle.tabucol(adj, k, start, 300, seed=2, ind=1, trace=True, check=True)
    col = start.astype(np.int64).copy()
    f = _f_from_edges(e, col)
    best = f
    for (v, c, d, t) in r["trace"]:
        if v < 0:
            continue
        # v is a conflicting vertex and c a different colour
        assert c != col[v] and np.any(adj[v][col == col[v]])
        # the reported delta is exact, and no unrestricted move (tabu or not) is better than the
        # best admissible one unless it is tabu: every strictly better move must be tabu and
        # must not reach below the best f (else aspiration would admit it)
        col2 = col.copy()
        col2[v] = c
        f2 = _f_from_edges(e, col2)
        assert f2 - f == d and t >= 1
        g = np.zeros((n, k), np.int64)
        np.add.at(g, (e[:, 0], col[e[:, 1]]), 1)
        np.add.at(g, (e[:, 1], col[e[:, 0]]), 1)
        gv = g[np.arange(n), col]
        for u in np.nonzero(gv > 0)[0]:
            for cc in range(k):
                if cc != col[u] and g[u, cc] - gv[u] < d:
                    assert f + g[u, cc] - gv[u] >= best  # not aspirated, hence tabu
        col, f = col2, f2
        best = min(best, f)
    assert best == r["best_f"]


def test_tabucol_determinism_and_seed_dependence():
    n, k = 60, 5
    adj = inputs.edges_to_adj(n, inputs.gnp(n, 0.4, seed=1))
    a = _run(adj, k, seed=1, iters=500)
    b = _run(adj, k, seed=1, iters=500)
    c = _run(adj, k, seed=2, iters=500)
    assert a["best_f"] == b["best_f"] and np.array_equal(a["best_col"], b["best_col"])
    assert not np.array_equal(a["best_col"], c["best_col"])


def test_tabucol_rejects_bad_colour():
    adj = inputs.edges_to_adj(5, inputs.cycle(5))
    with pytest.raises(RuntimeError):
        oracle.tabucol(adj, 2, np.array([0, 1, 2, 0, 1], np.int16), 10, seed=0, ind=0)
