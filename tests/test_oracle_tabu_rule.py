"""Pins of the oracle's tabu rule itself: tenure, aspiration, the no-move case and the tie pick.

The outcome pins elsewhere (brute-force chromatic numbers, closed forms, recounts) fix where a
search ends and that every move's delta is exact. They do not fix the rule that decides which
move is taken. Here an independent plain-Python replay of TabuCol (section "Adaptations of the
algorithm for the vertex coloring problem"; alpha = 0.6 from Table params-COL) and of the
weighted search's vertex freeze (section "Parallel iterated feasible and infeasible Tabu
Search", tenure U{0..9} + 0.2 |V|) keeps its own tabu lists, recomputes every admissible move
from the conflict table and draws the tie index from the known-answer-pinned Philox generator.
The oracle's traces must equal the replay move by move. Each replay can also be run with a
plausible mistake planted (tenure from f before the move, expiry at it + tt, aspiration with
<=, the last tie instead of the j-th, column-major tie order, a re-tabued pair keeping the later
of its two expiries instead of the new one); every such variant must disagree
with the oracle on these cases, which shows that the comparison can see that mistake.

CPU only; the oracle is the code under test.
"""
import numpy as np
import pytest

import oracle
from paper_2109_05948_gb300 import inputs

TWO32 = 1 << 32


def _below(r, m):
    """Uniform integer in [0, m): the high word of r * m (the rule stated for every draw)."""
    return (int(r) * int(m)) >> 32


def _gamma(adj, col, k):
    n = adj.shape[0]
    g = np.zeros((n, k), np.int64)
    for c in range(k):
        g[:, c] = adj[:, col == c].sum(1)
    return g


def replay_tabucol(adj, k, start, iters, seed, ind, gen=0, L_max=9, an=6, ad=10, variant=None):
    """TabuCol restated from the rule: the neighbourhood is every (v, c) with v conflicting and
    c != col v; a move is admissible when it is not tabu (tabu_until[v][c] <= it) or when it
    reaches below the best f seen (aspiration); the smallest delta wins, ties broken by the
    j-th admissible minimum in row-major (v, c) order with j = floor(r0 T / 2^32); the old
    colour of the moved vertex is tabu until it + 1 + floor(r1 (L_max + 1) / 2^32) +
    floor(an f_after / ad); with no admissible move the iteration passes; the search stops at
    f = 0. Returns (trace, best_f, best_col, moves, stats)."""
    adj = np.asarray(adj, np.int64)
    n = adj.shape[0]
    col = np.asarray(start, np.int64).copy()
    tabu_until = np.zeros((n, k), np.int64)
    g = _gamma(adj, col, k)
    f = int(g[np.arange(n), col].sum() // 2)
    best_f, best_col, moves = f, col.copy(), 0
    trace = []
    stats = dict(aspirated=0, blocked=0, ties=0, nomove=0, retabu=0)
    for it in range(iters):
        if f == 0:
            break
        r = oracle.draw(seed, it, gen, ind, oracle.TAG_TABU)
        g0 = g[np.arange(n), col]
        cand = []  # admissible moves in row-major order
        blocked = None  # smallest delta among the moves the tabu list refused
        for v in range(n):
            if g0[v] == 0:
                continue
            for c in range(k):
                if c == col[v]:
                    continue
                d = int(g[v, c] - g0[v])
                tabu = tabu_until[v, c] > it
                if variant == "aspiration_le":
                    asp = f + d <= best_f
                else:
                    asp = f + d < best_f
                if not tabu or asp:
                    cand.append((d, v, c, tabu))
                elif blocked is None or d < blocked:
                    blocked = d
        if not cand:
            trace.append((-1, -1, 0, 0))
            stats["nomove"] += 1
            continue
        dmin = min(x[0] for x in cand)
        ties = [x for x in cand if x[0] == dmin]
        T = len(ties)
        if variant == "tie_column_major":
            ties.sort(key=lambda x: (x[2], x[1]))
        j = _below(r[0], T)
        if variant == "tie_last":
            j = T - 1 - j
        d, v, c, was_tabu = ties[j]
        stats["aspirated"] += int(was_tabu)
        stats["ties"] += int(T > 1)
        stats["blocked"] += int(blocked is not None and blocked < dmin)
        old = int(col[v])
        f_before = f
        col[v] = c
        nb = np.nonzero(adj[v])[0]
        g[nb, old] -= 1
        g[nb, c] += 1
        f += d
        f_ten = f_before if variant == "tenure_from_f_before" else f
        tt = _below(r[1], L_max + 1) + (an * f_ten) // ad
        stats["retabu"] += int(tabu_until[v, old] > it)
        until = it + (0 if variant == "expiry_at_it_plus_tt" else 1) + tt
        if variant == "retabu_keeps_later_expiry":
            until = max(until, tabu_until[v, old])
        tabu_until[v, old] = until
        moves += 1
        if f < best_f:
            best_f, best_col = f, col.copy()
        trace.append((v, c, d, T))
    return np.array(trace, np.int64).reshape(-1, 4), best_f, best_col, moves, stats


def _oracle_run(adj, k, start, iters, seed, ind, gen=0, L_max=9, alpha=(6, 10)):
    return oracle.tabucol(adj, k, start, iters, seed=seed, ind=ind, gen=gen, L_max=L_max, alpha=alpha, trace=True)


# Cases that between them take every branch of the rule: aspirated moves, strictly better moves
# blocked by the tabu list, tied minima, iterations with no admissible move, and a vertex leaving a
# colour that is still tabu for it (an aspirated move into it happened first).
CASES = [
    dict(n=30, p=0.3, k=4, iters=400, seed=11, ind=3, L_max=9, alpha=(6, 10)),
    dict(n=24, p=0.5, k=5, iters=400, seed=12, ind=0, L_max=9, alpha=(6, 10)),
    dict(n=18, p=0.4, k=3, iters=300, seed=13, ind=7, L_max=9, alpha=(60, 10)),  # long tenures: no-move iterations
    dict(n=40, p=0.15, k=3, iters=500, seed=14, ind=1, L_max=3, alpha=(6, 10)),
    dict(n=40, p=0.5, k=4, iters=400, seed=35, ind=1, L_max=9, alpha=(6, 10)),  # two re-tabued pairs
    dict(n=60, p=0.5, k=5, iters=300, seed=33, ind=1, L_max=9, alpha=(6, 10)),
    dict(n=40, p=0.5, k=4, iters=500, seed=32, ind=1, L_max=9, alpha=(20, 10)),  # a re-tabu shortens a tenure
]


def _case_inputs(cs):
    e = inputs.gnp(cs["n"], cs["p"], seed=cs["seed"])
    adj = inputs.edges_to_adj(cs["n"], e)
    start = inputs.random_colorings(1, cs["n"], cs["k"], seed=cs["seed"])[0]
    return adj, start


def test_tabucol_hand_worked_six_vertex_case():
    """Four iterations worked out by hand from the rule (L_max = 0, so the tenure is
    floor(0.6 f_after) and no tie arises).

    Edges 0-5, 1-4, 2-3, 2-4, 3-4, 3-5, 4-5; k = 2; start colouring (1, 1, 0, 1, 1, 1).
    it 0: conflicting edges 0-5, 1-4, 3-4, 3-5, 4-5, f = 5. Moves to colour 0 change f by
          -1 (v0), -1 (v1), -1 (v3), -2 (v4), -3 (v5): v5 -> 0, f = 2, tenure floor(1.2) = 1,
          (5, 1) tabu until 0 + 1 + 1 = 2.
    it 1: conflicts 1-4, 3-4. v1 -> 0 gives -1, v3 -> 0 gives +1, v4 -> 0 gives 0: v1 -> 0,
          f = 1 (the best so far), tenure floor(0.6) = 0, (1, 1) tabu until 2.
    it 2: only 3-4 conflicts. v3 -> 0 gives +1, v4 -> 0 gives +2: v3 -> 0, f = 2, tenure
          floor(1.2) = 1, (3, 1) tabu until 2 + 1 + 1 = 4.
    it 3: conflicts 2-3, 3-5. v3 -> 1 would give -1 but is tabu (4 > 3) and not aspirated
          (f - 1 = 1 is not below the best 1); v2 -> 1 gives 0, v5 -> 1 gives +1: v2 -> 1.
    A tenure taken from f before the move (floor(0.6) = 0 at it 2), an expiry at it + tt, or an
    aspiration with <= would each let v3 -> 1 through at it 3.
    """
    n, k = 6, 2
    e = np.array([[0, 5], [1, 4], [2, 3], [2, 4], [3, 4], [3, 5], [4, 5]], np.int32)
    adj = inputs.edges_to_adj(n, e)
    start = np.array([1, 1, 0, 1, 1, 1], np.int16)
    r = _oracle_run(adj, k, start, 4, seed=5, ind=0, L_max=0)
    expect = [(5, 0, -3, 1), (1, 0, -1, 1), (3, 0, 1, 1), (2, 1, 0, 1)]
    assert [tuple(int(x) for x in row) for row in r["trace"]] == expect
    assert r["best_f"] == 1 and r["moves"] == 4
    assert list(r["best_col"]) == [1, 0, 0, 1, 1, 0]  # the colouring after it 1
    # the planted mistakes change iteration 3 of this case
    for variant in ("tenure_from_f_before", "expiry_at_it_plus_tt", "aspiration_le"):
        tr = replay_tabucol(adj, k, start, 4, seed=5, ind=0, L_max=0, variant=variant)[0]
        assert tuple(tr[3]) != expect[3], variant


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_tabucol_trace_equals_independent_replay(ci):
    cs = CASES[ci]
    adj, start = _case_inputs(cs)
    r = _oracle_run(adj, cs["k"], start, cs["iters"], cs["seed"], cs["ind"], L_max=cs["L_max"], alpha=cs["alpha"])
    tr, bf, bc, mv, stats = replay_tabucol(adj, cs["k"], start, cs["iters"], cs["seed"], cs["ind"],
                                           L_max=cs["L_max"], an=cs["alpha"][0], ad=cs["alpha"][1])
    assert tr.shape == r["trace"].shape
    assert np.array_equal(tr, r["trace"])
    assert bf == r["best_f"] and mv == r["moves"]
    assert np.array_equal(bc, r["best_col"])
    if ci == 2:
        assert stats["nomove"] > 0


def test_replay_cases_take_every_branch_of_the_rule():
    tot = dict(aspirated=0, blocked=0, ties=0, nomove=0, retabu=0)
    for cs in CASES:
        adj, start = _case_inputs(cs)
        st = replay_tabucol(adj, cs["k"], start, cs["iters"], cs["seed"], cs["ind"], L_max=cs["L_max"],
                            an=cs["alpha"][0], ad=cs["alpha"][1])[4]
        for key in tot:
            tot[key] += st[key]
    assert all(v > 0 for v in tot.values()), tot


@pytest.mark.parametrize("variant", ["tenure_from_f_before", "expiry_at_it_plus_tt", "aspiration_le", "tie_last",
                                     "tie_column_major", "retabu_keeps_later_expiry"])
def test_each_planted_rule_mistake_is_seen(variant):
    seen = False
    for cs in CASES:
        adj, start = _case_inputs(cs)
        r = _oracle_run(adj, cs["k"], start, cs["iters"], cs["seed"], cs["ind"], L_max=cs["L_max"],
                        alpha=cs["alpha"])
        tr = replay_tabucol(adj, cs["k"], start, cs["iters"], cs["seed"], cs["ind"], L_max=cs["L_max"],
                            an=cs["alpha"][0], ad=cs["alpha"][1], variant=variant)[0]
        if tr.shape != r["trace"].shape or not np.array_equal(tr, r["trace"]):
            seen = True
            break
    assert seen, f"the replay with '{variant}' still equals the oracle"


# ------------------------------------------------------------------------------------------------
# weighted search: vertex freeze
# ------------------------------------------------------------------------------------------------
def _wvcp_g(adj, w, k, col, fscale, phi):
    mx = np.zeros(k, np.int64)
    np.maximum.at(mx, col, w)
    conf = int(np.triu(adj * (col[:, None] == col[None, :]), 1).sum())
    return fscale * int(mx.sum()) + phi * conf, int(mx.sum()), conf


def replay_wvcp(adj, w, k, start, iters, phi, seed, ind, gen=0, fscale=1, L_max=9, an=2, ad=10, variant=None):
    """The weighted search restated from its definition: every one-move (v, c != col v) is
    scored by recomputing g = fscale * sum_c max_{v in V_c} w_v + phi * #conflicting edges; a
    move is admissible when v is not frozen (frozen_until[v] <= it) or it reaches below the best
    g; the smallest delta wins with the same tie rule as TabuCol; the moved vertex is frozen
    until it + 1 + floor(r1 (L_max + 1) / 2^32) + floor(an n / ad)."""
    adj = np.asarray(adj, np.int64)
    w = np.asarray(w, np.int64)
    n = adj.shape[0]
    col = np.asarray(start, np.int64).copy()
    frozen = np.zeros(n, np.int64)
    g, _, _ = _wvcp_g(adj, w, k, col, fscale, phi)
    best_g, moves, trace = g, 0, []
    stats = dict(aspirated=0, blocked=0, ties=0)
    base = (an * n) // ad
    for it in range(iters):
        r = oracle.draw(seed, it, gen, ind, oracle.TAG_TABU)
        cand, blocked = [], None
        for v in range(n):
            for c in range(k):
                if c == col[v]:
                    continue
                col2 = col.copy()
                col2[v] = c
                d = _wvcp_g(adj, w, k, col2, fscale, phi)[0] - g
                fr = frozen[v] > it
                if not fr or g + d < best_g:
                    cand.append((d, v, c, fr))
                elif blocked is None or d < blocked:
                    blocked = d
        if not cand:
            trace.append((-1, -1, 0, 0))
            continue
        dmin = min(x[0] for x in cand)
        ties = [x for x in cand if x[0] == dmin]
        j = _below(r[0], len(ties))
        d, v, c, fr = ties[j]
        stats["aspirated"] += int(fr)
        stats["blocked"] += int(blocked is not None and blocked < dmin)
        stats["ties"] += int(len(ties) > 1)
        col[v] = c
        g += d
        tt = _below(r[1], L_max + 1) + (base if variant != "freeze_from_alpha_f" else 0)
        frozen[v] = it + (0 if variant == "freeze_at_it_plus_tt" else 1) + tt
        moves += 1
        best_g = min(best_g, g)
        trace.append((v, c, d, len(ties)))
    return np.array(trace, np.int64).reshape(-1, 4), best_g, moves, stats


WCASES = [
    dict(n=14, p=0.4, k=4, iters=150, phi=20, seed=21, ind=2),
    dict(n=12, p=0.5, k=5, iters=150, phi=3, seed=22, ind=5),
]


def _wcase_inputs(cs):
    e = inputs.gnp(cs["n"], cs["p"], seed=cs["seed"])
    adj = inputs.edges_to_adj(cs["n"], e)
    w = inputs.weights(cs["n"], seed=cs["seed"], hi=12)  # few weight levels: ties in the objective
    start = inputs.random_colorings(1, cs["n"], cs["k"], seed=cs["seed"])[0]
    return adj, w, start


@pytest.mark.parametrize("ci", range(len(WCASES)))
def test_wvcp_trace_equals_independent_replay(ci):
    cs = WCASES[ci]
    adj, w, start = _wcase_inputs(cs)
    r = oracle.wvcp_tabu(adj, w, cs["k"], start, cs["iters"], cs["phi"], seed=cs["seed"], ind=cs["ind"], trace=True)
    tr, bg, mv, st = replay_wvcp(adj, w, cs["k"], start, cs["iters"], cs["phi"], cs["seed"], cs["ind"])
    assert np.array_equal(tr, r["trace"][: len(tr)]) and len(tr) == cs["iters"]
    assert bg == r["best_g"] and mv == r["moves"]


def test_wvcp_replay_cases_take_every_branch():
    tot = dict(aspirated=0, blocked=0, ties=0)
    for cs in WCASES:
        adj, w, start = _wcase_inputs(cs)
        st = replay_wvcp(adj, w, cs["k"], start, cs["iters"], cs["phi"], cs["seed"], cs["ind"])[3]
        for key in tot:
            tot[key] += st[key]
    assert all(v > 0 for v in tot.values()), tot


@pytest.mark.parametrize("variant", ["freeze_at_it_plus_tt", "freeze_from_alpha_f"])
def test_wvcp_planted_freeze_mistake_is_seen(variant):
    cs = WCASES[0]
    adj, w, start = _wcase_inputs(cs)
    r = oracle.wvcp_tabu(adj, w, cs["k"], start, cs["iters"], cs["phi"], seed=cs["seed"], ind=cs["ind"], trace=True)
    tr = replay_wvcp(adj, w, cs["k"], start, cs["iters"], cs["phi"], cs["seed"], cs["ind"], variant=variant)[0]
    assert not np.array_equal(tr, r["trace"])
