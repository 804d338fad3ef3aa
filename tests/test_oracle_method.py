"""Pins of the oracle's GPX, distance, pool update, KNN, scorer, Adam, WVCP and memetic loop
against properties fixed by the paper's definitions and by mathematics (CPU only)."""
import itertools

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import oracle
from paper_2109_05948_gb300 import inputs


# ------------------------------------------------------------------------------------------------
# GPX
# ------------------------------------------------------------------------------------------------
def _classes_by_size(A, k):
    sizes = np.bincount(A, minlength=k)
    return sorted(range(k), key=lambda c: (-sizes[c], c)), sizes


def test_gpx_identical_parents_relabel_by_decreasing_size():
    n, k = 50, 6
    A = inputs.random_colorings(1, n, k, seed=3)[0]
    child = oracle.gpx(k, A, A, seed=1, child_id=0)
    order, sizes = _classes_by_size(A, k)
    expect = np.empty(n, np.int16)
    for lab, c in enumerate(order):
        expect[A == c] = lab
    assert np.array_equal(child, expect)


def test_gpx_relabelled_parent_gives_same_partition():
    n, k = 60, 5
    A = inputs.random_colorings(1, n, k, seed=4)[0]
    sigma = np.random.default_rng(0).permutation(k)
    child = oracle.gpx(k, A, sigma[A].astype(np.int16), seed=1, child_id=3)
    # same partition: a bijection between labels
    pairs = set(zip(A.tolist(), child.tolist()))
    assert len(pairs) == len(set(A.tolist())) == len(set(child.tolist()))


def test_gpx_first_two_steps_and_leftovers():
    n, k = 80, 6
    A, B = inputs.random_colorings(2, n, k, seed=5)
    seed, cid, gen = 7, 11, 2
    child = oracle.gpx(k, A, B, seed=seed, child_id=cid, gen=gen)
    assert child.min() >= 0 and child.max() < k
    # step 0 takes the largest class of A (smallest colour on ties) with label 0
    a0 = _classes_by_size(A, k)[0][0]
    assert np.all(child[A == a0] == 0)
    # step 1 takes the largest class of B among the remaining vertices, label 1
    rem = A != a0
    sizes_b = np.bincount(B[rem], minlength=k)
    b1 = int(np.argmax(sizes_b))
    assert np.all(child[rem & (B == b1)] == 1)
    # every child class is a union of parent-class pieces: each label l < k that comes from an
    # inherited class is a subset of one class of A (even l) or of B (odd l), plus leftovers whose
    # labels come from the GPX Philox stream
    taken = np.zeros(n, bool)
    for lab in range(k):
        P = A if lab % 2 == 0 else B
        cnt = np.bincount(P[~taken], minlength=k)
        if cnt.max() == 0:
            break
        c = int(np.argmax(cnt))
        sel = (~taken) & (P == c)
        assert np.all(child[sel] == lab)
        taken |= sel
    for v in np.nonzero(~taken)[0]:
        r = oracle.draw(seed, int(v), gen, cid, oracle.TAG_GPX)
        assert child[v] == (int(r[0]) * k) >> 32


# ------------------------------------------------------------------------------------------------
# distance
# ------------------------------------------------------------------------------------------------
def _exact_distance(A, B, k):
    M = np.zeros((k, k), np.int64)
    np.add.at(M, (A, B), 1)
    r, c = linear_sum_assignment(-M)
    return len(A) - int(M[r, c].sum())


@pytest.mark.parametrize("n,k,seed", [(12, 3, 0), (20, 4, 1), (30, 5, 2), (40, 6, 3), (9, 6, 4)])
def test_distance_exact_against_brute_force_matchings(n, k, seed):
    """oracle.distance_exact is n minus the best one-to-one class matching: checked against every
    permutation of the k classes, with the overlaps counted vertex by vertex."""
    import itertools

    A, B = inputs.random_colorings(2, n, k, seed=seed)
    best = 0
    for perm in itertools.permutations(range(k)):
        best = max(best, sum(1 for v in range(n) if perm[A[v]] == B[v]))
    assert oracle.distance_exact(k, A, B) == n - best
    assert oracle.distance_exact(k, A, B) == oracle.distance_exact(k, B, A)
    assert oracle.distance(k, A, B) <= oracle.distance_exact(k, A, B)


def test_distance_exact_relabel_and_recolour():
    n, k = 150, 9
    A = inputs.random_colorings(1, n, k, seed=7)[0]
    sigma = np.random.default_rng(3).permutation(k)
    B = sigma[A].astype(np.int16)
    assert oracle.distance_exact(k, A, B) == 0
    # recolouring m vertices of a partition with classes of at least 2 m + 1 vertices costs exactly m
    A = np.repeat(np.arange(k), n // k + 1)[:n].astype(np.int16)
    B = A.copy()
    idx = np.random.default_rng(4).choice(n, 5, replace=False)
    B[idx] = (B[idx] + 1) % k
    assert oracle.distance_exact(k, A, B) == 5


def test_distance_relabel_is_zero_and_symmetric():
    n, k = 100, 8
    A, B = inputs.random_colorings(2, n, k, seed=6)
    sigma = np.random.default_rng(1).permutation(k)
    assert oracle.distance(k, A, sigma[A].astype(np.int16)) == 0
    assert oracle.distance(k, A, A) == 0
    assert oracle.distance(k, A, B) == oracle.distance(k, B, A)


@pytest.mark.parametrize("seed", range(6))
def test_distance_lower_bound_of_exact(seed):
    n, k = 90, 7
    A, B = inputs.random_colorings(2, n, k, seed=10 + seed)
    assert 0 <= oracle.distance(k, A, B) <= _exact_distance(A, B, k)


@pytest.mark.parametrize("moves", [1, 3, 9])
def test_distance_exact_when_matching_injective(moves):
    n, k = 120, 6
    rng = np.random.default_rng(moves)
    A = np.repeat(np.arange(k), n // k).astype(np.int16)
    rng.shuffle(A)
    B = np.random.default_rng(2).permutation(k)[A].astype(np.int16)
    idx = rng.choice(n, moves, replace=False)
    B[idx] = (B[idx] + 1) % k
    d = oracle.distance(k, A, B)
    assert d == _exact_distance(A, B, k) == moves


# ------------------------------------------------------------------------------------------------
# pool update and parent matching
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(4))
def test_pool_update_greedy_characterisation(seed):
    p, n = 30, 50
    rng = np.random.default_rng(seed)
    m = 2 * p
    D = rng.integers(0, 12, size=(m, m))
    D = np.triu(D, 1)
    D = (D + D.T).astype(np.int16)
    fit = rng.integers(0, 20, size=m).astype(np.int64)
    sel = oracle.pool_update(p, n, fit, D)
    assert len(set(sel.tolist())) == p
    order = np.lexsort((np.arange(m), fit))  # by f, ties by index (the population first)
    pos = {int(x): i for i, x in enumerate(order)}
    spaced = []
    for x in sel:
        if all(10 * D[x, y] > n for y in spaced):
            spaced.append(int(x))
        else:
            break
    # admitted members are spaced and appear in fitness order
    assert [pos[x] for x in spaced] == sorted(pos[x] for x in spaced)
    last = pos[spaced[-1]]
    for t in range(last):
        x = int(order[t])
        if x not in spaced:  # rejected: too close to an earlier admitted member
            assert any(10 * D[x, y] <= n for y in spaced if pos[y] < t)
    # the rest (when fewer than p are spaced) are the best remaining by the same order
    rest = [int(x) for x in sel[len(spaced):]]
    remaining = [int(x) for x in order if int(x) not in spaced]
    if rest:
        # no candidate after the last spaced one could have been admitted
        for t in range(last + 1, m):
            x = int(order[t])
            assert any(10 * D[x, y] <= n for y in spaced)
        assert rest == remaining[: len(rest)]


def test_knn_matches_library_sort():
    p, K = 40, 7
    rng = np.random.default_rng(3)
    D = rng.integers(0, 9, size=(p, p))
    D = (np.triu(D, 1) + np.triu(D, 1).T).astype(np.int16)
    nbr = oracle.knn(D, K)
    for i in range(p):
        js = np.array([j for j in range(p) if j != i])
        o = js[np.argsort(D[i, js], kind="stable")][:K]
        assert list(nbr[i]) == list(o)


# ------------------------------------------------------------------------------------------------
# scorer
# ------------------------------------------------------------------------------------------------
def test_scorer_finite_differences():
    dims = oracle.ScorerDims(n=10, d0=4, d=6, nl=3)
    k = 3
    th = oracle.scorer_init(dims, seed=5)
    th += np.random.default_rng(0).normal(0, 0.3, th.shape)  # move away from tiny init values
    cols = inputs.random_colorings(3, 10, k, seed=2)
    y = np.array([0.3, -1.0, 2.0])
    loss, g, _ = oracle.scorer_loss_grad(dims, k, th, cols, y)
    h = 1e-6
    num = np.zeros_like(th)
    for i in range(th.size):
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        num[i] = (oracle.scorer_loss_grad(dims, k, tp, cols, y)[0] - oracle.scorer_loss_grad(dims, k, tm, cols, y)[0]) / (2 * h)
    err = np.abs(num - g) / np.maximum(1e-6, np.abs(g) + np.abs(num))
    assert np.max(np.abs(num - g)) < 1e-6 * max(1.0, np.abs(g).max()) * 10
    assert np.median(err) < 1e-6


def test_scorer_colour_permutation_invariance():
    dims = oracle.ScorerDims(n=30, d0=8, d=16, nl=3)
    k = 5
    th = oracle.scorer_init(dims, seed=1)
    cols = inputs.random_colorings(4, 30, k, seed=9)
    sigma = np.random.default_rng(4).permutation(k)
    a = oracle.scorer_forward(dims, k, th, cols)
    b = oracle.scorer_forward(dims, k, th, sigma[cols].astype(np.int16))
    assert np.allclose(a, b, rtol=0, atol=1e-12)
    # not invariant to moving one vertex between classes
    c2 = cols.copy()
    c2[:, 0] = (c2[:, 0] + 1) % k
    assert not np.allclose(a, oracle.scorer_forward(dims, k, th, c2))


def test_scorer_closed_form_positive_regime():
    """With every weight and bias positive the network is linear and, because each vertex sits in
    exactly one class, out = bh + wh . (b3 + (b2 + (b1 + m0 (L1 + G1)) (L2 + G2)) (L3 + G3)) with
    m0 = b0 + sum(E) / k, whatever the colouring."""
    n, d0, d, k = 20, 4, 5, 3
    dims = oracle.ScorerDims(n=n, d0=d0, d=d, nl=3)
    rng = np.random.default_rng(7)
    th = rng.uniform(0.01, 0.2, dims.nparams())
    o = dims.offsets()
    get = lambda name: th[o[name][0]:o[name][0] + int(np.prod(o[name][1]))].reshape(o[name][1])
    m = get("b0") + get("E").sum(0) / k
    for l in (1, 2, 3):
        m = get(f"b{l}") + m @ (get(f"lam{l}") + get(f"gam{l}"))
    expect = get("bh")[0] + m @ get("wh")
    cols = inputs.random_colorings(3, n, k, seed=1)
    assert np.allclose(oracle.scorer_forward(dims, k, th, cols), expect, rtol=1e-12)


def test_scorer_zero_weights_closed_form():
    n, d0, d, k = 12, 4, 6, 4
    dims = oracle.ScorerDims(n=n, d0=d0, d=d, nl=3)
    th = oracle.scorer_init(dims, seed=3)
    o = dims.offsets()
    for l in (1, 2, 3):
        for nm in (f"lam{l}", f"gam{l}"):
            th[o[nm][0]:o[nm][0] + int(np.prod(o[nm][1]))] = 0.0
    b3 = th[o["b3"][0]:o["b3"][0] + d]
    wh = th[o["wh"][0]:o["wh"][0] + d]
    expect = th[o["bh"][0]] + np.where(b3 > 0, b3, 0.2 * b3) @ wh
    cols = inputs.random_colorings(2, n, k, seed=2)
    assert np.allclose(oracle.scorer_forward(dims, k, th, cols), expect, rtol=1e-13)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(0)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    m, v = np.zeros(50), np.zeros(50)
    th0 = th.copy()
    oracle.adam_step(th, m, v, g, 1, 1e-3)
    assert np.allclose(th, th0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_scorer_training_reduces_loss():
    n, k, p = 24, 3, 40
    dims = oracle.ScorerDims(n=n, d0=8, d=16, nl=3)
    th = oracle.scorer_init(dims, seed=2)
    am, av = np.zeros_like(th), np.zeros_like(th)
    cols = inputs.random_colorings(p, n, k, seed=5)
    # a learnable target: the size of class 0
    f = np.bincount(np.nonzero(cols == 0)[0], minlength=p).astype(np.int64)
    y = (f - f.mean()) / f.std()
    l0 = oracle.scorer_loss_grad(dims, k, th, cols, y)[0]
    _, t = oracle.scorer_train(dims, k, th, am, av, 0, cols, f, epochs=30, b=10, lr=1e-2, seed=1, gen=0)
    assert t == 30 * 4
    assert oracle.scorer_loss_grad(dims, k, th, cols, y)[0] < 0.5 * l0


# ------------------------------------------------------------------------------------------------
# WVCP
# ------------------------------------------------------------------------------------------------
def test_wvcp_score_definition():
    n, k = 40, 7
    adj = inputs.edges_to_adj(n, inputs.gnp(n, 0.3, seed=1))
    w = inputs.weights(n, seed=1)
    col = inputs.random_colorings(1, n, k, seed=3)[0]
    L = oracle.lib()
    conf = np.zeros(1, np.int64)
    f = L.oracle_wvcp_score(n, oracle._ptr(adj), oracle._ptr(w), k, oracle._ptr(col), oracle._ptr(conf))
    assert f == sum(int(w[col == c].max()) for c in range(k) if np.any(col == c))
    ones = np.ones(n, np.int32)
    assert L.oracle_wvcp_score(n, oracle._ptr(adj), oracle._ptr(ones), k, oracle._ptr(col), None) == len(set(col.tolist()))
    assert conf[0] == oracle.gamma(adj, k, col)[1]


def _wvcp_greedy(adj, w, seed, ind=0):
    n = adj.shape[0]
    col = np.zeros(n, np.int16)
    used = oracle.lib().oracle_wvcp_greedy(n, oracle._ptr(adj), oracle._ptr(w), seed, ind, oracle._ptr(col))
    return col, used


def _wvcp_tabu(adj, w, k, col, iters, phi, seed, ind=0, check=True, L_max=9, alpha=(2, 10)):
    n = adj.shape[0]
    best = np.zeros(n, np.int16)
    bg, fc, mv = np.zeros(1, np.int64), np.zeros(2, np.int64), np.zeros(1, np.int64)
    rc = oracle.lib().oracle_wvcp_tabu(n, oracle._ptr(adj), oracle._ptr(w), k, oracle._ptr(col), iters, L_max,
                                       alpha[0], alpha[1], phi, seed, ind, 0, oracle._ptr(best), oracle._ptr(bg),
                                       oracle._ptr(fc), oracle._ptr(mv), None, 1 if check else 0)
    assert rc == 0
    return best, int(bg[0]), int(fc[0]), int(fc[1]), int(mv[0])


def test_wvcp_greedy_is_legal_and_ordered():
    n = 60
    e = inputs.gnp(n, 0.4, seed=2)
    adj = inputs.edges_to_adj(n, e)
    w = inputs.weights(n, seed=2)
    col, used = _wvcp_greedy(adj, w, seed=4)
    assert int(np.sum(col[e[:, 0]] == col[e[:, 1]])) == 0
    assert set(col.tolist()) == set(range(used))
    deg = adj.sum(1).astype(np.int64)
    w = w.astype(np.int64)
    first = sorted(range(n), key=lambda v: (-w[v], -deg[v], v))[0]
    assert col[first] == 0


def _wvcp_brute(n, edges, w, k):
    best = None
    for cols in itertools.product(range(k), repeat=n):
        c = np.array(cols)
        if np.any(c[edges[:, 0]] == c[edges[:, 1]]):
            continue
        f = sum(int(w[c == q].max()) for q in range(k) if np.any(c == q))
        best = f if best is None else min(best, f)
    return best


@pytest.mark.parametrize("gseed", [1, 2, 3])
def test_wvcp_tabu_reaches_brute_force_optimum(gseed):
    n = 7
    e = inputs.gnp(n, 0.5, seed=gseed)
    adj = inputs.edges_to_adj(n, e)
    w = inputs.weights(n, seed=gseed)
    col, used = _wvcp_greedy(adj, w, seed=gseed)
    k = used
    phi = 2 * int(w.max())
    best, bg, bf, bc, _ = _wvcp_tabu(adj, w, k, col, 2000, phi, seed=gseed)
    assert bc == 0 and bg == bf == _wvcp_brute(n, e, w, k)


def test_wvcp_tabu_check_mode_and_recount():
    n = 50
    e = inputs.gnp(n, 0.5, seed=5)
    adj = inputs.edges_to_adj(n, e)
    w = inputs.weights(n, seed=5)
    col, used = _wvcp_greedy(adj, w, seed=1)
    start = inputs.random_colorings(1, n, used, seed=3)[0]  # an illegal start
    phi = 2 * int(w.max())
    best, bg, bf, bc, mv = _wvcp_tabu(adj, w, used, start, 500, phi, seed=2, check=True)
    conf = int(np.sum(best[e[:, 0]] == best[e[:, 1]]))
    f = sum(int(w[best == q].max()) for q in range(used) if np.any(best == q))
    assert (bf, bc, bg) == (f, conf, f + phi * conf)
    assert mv > 0


def _wvcp_case(n, p, seed):
    e = inputs.gnp(n, p, seed=seed)
    return e, inputs.edges_to_adj(n, e), inputs.weights(n, seed=seed)


@pytest.mark.parametrize("scale", [2, 256])
def test_wvcp_scaled_objective_moves_like_the_unscaled_one(scale):
    """g = s f + (s phi) c is s times f + phi c, so every delta scales by s and the search takes the
    same moves (check mode recounts f, c and g after each of them)."""
    n = 45
    e, adj, w = _wvcp_case(n, 0.4, 6)
    col, used = _wvcp_greedy(adj, w, seed=6)
    start = inputs.random_colorings(1, n, used, seed=8)[0]
    phi = 37
    a = oracle.wvcp_tabu(adj, w, used, start, 400, phi, seed=3, ind=1, trace=True, check=True)
    b = oracle.wvcp_tabu(adj, w, used, start, 400, scale * phi, seed=3, ind=1, fscale=scale, trace=True, check=True)
    assert np.array_equal(a["trace"][:, :2], b["trace"][:, :2]) and np.array_equal(a["trace"][:, 3], b["trace"][:, 3])
    assert np.array_equal(a["trace"][:, 2] * scale, b["trace"][:, 2])
    assert (a["f"], a["c"], a["moves"]) == (b["f"], b["c"], b["moves"]) and b["best_g"] == scale * a["best_g"]
    assert np.array_equal(a["best_col"], b["best_col"])


def test_wvcp_iterated_single_search_is_the_last_run_setting():
    """With one search, Algorithm 2 is one tabu search at phi = phi_last (generation 16 gen)."""
    n = 40
    e, adj, w = _wvcp_case(n, 0.5, 2)
    col, used = _wvcp_greedy(adj, w, seed=2)
    start = inputs.random_colorings(1, n, used, seed=4)[0]
    phi_last = 2 * int(w.max())
    it = oracle.wvcp_iterated(adj, w, used, start, 300, 1, 1, 5, phi_last, seed=7, ind=3, gen=2)
    ref = oracle.wvcp_tabu(adj, w, used, start, 300, phi_last, seed=7, ind=3, gen=32)
    assert list(it["phi"]) == [phi_last] and (it["fc"][0, 0], it["fc"][0, 1]) == (ref["f"], ref["c"])
    if ref["c"] == 0:
        assert it["best_f"] == ref["f"] and np.array_equal(it["best_col"], ref["best_col"])
    else:
        assert it["best_f"] == -1


@pytest.mark.parametrize("gseed", [1, 3])
def test_wvcp_iterated_schedule_and_best_legal(gseed):
    """phi halves after a search whose best colouring is legal and doubles otherwise (floor, at least
    1), the last search uses phi_last, and S' is the legal search result with the smallest f."""
    n = 60
    e, adj, w = _wvcp_case(n, 0.5, gseed)
    col, used = _wvcp_greedy(adj, w, seed=gseed)
    start = inputs.random_colorings(1, n, used, seed=gseed + 10)[0]
    fscale, max_ls = 256, 10
    phi0 = (fscale * used * int(w.max()) + n) // (2 * n)
    phi_last = fscale * 2 * int(w.max())
    r = oracle.wvcp_iterated(adj, w, used, start, 150, max_ls, fscale, phi0, phi_last, seed=gseed, ind=0, gen=1)
    phis, fcs = r["phi"], r["fc"]
    assert phis[0] == phi0 and phis[-1] == phi_last
    for t in range(max_ls - 2):
        legal = fcs[t, 1] == 0
        assert phis[t + 1] == (max(1, phis[t] // 2) if legal else 2 * phis[t])
    legal_f = [int(f) for f, c in fcs if c == 0]
    assert r["best_f"] == (min(legal_f) if legal_f else -1)
    if legal_f:
        b = r["best_col"]
        assert int(np.sum(b[e[:, 0]] == b[e[:, 1]])) == 0
        assert sum(int(w[b == q].max()) for q in range(used) if np.any(b == q)) == r["best_f"]


@pytest.mark.parametrize("gseed", [1, 2])
def test_wvcp_iterated_reaches_brute_force_optimum(gseed):
    n = 7
    e = inputs.gnp(n, 0.5, seed=gseed)
    adj = inputs.edges_to_adj(n, e)
    w = inputs.weights(n, seed=gseed)
    col, used = _wvcp_greedy(adj, w, seed=gseed)
    r = oracle.wvcp_iterated(adj, w, used, col, 300, 10, 256, (256 * used * int(w.max()) + n) // (2 * n),
                             256 * 2 * int(w.max()), seed=gseed, ind=0)
    assert r["best_f"] == _wvcp_brute(n, e, w, used)


# ------------------------------------------------------------------------------------------------
# memetic generation (Algorithm 1)
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("use_scorer", [0, 1])
def test_memetic_generation_invariants(use_scorer):
    n, k, p, K = 40, 4, 16, 4
    e, _ = inputs.planted(n, k, 0.4, seed=3)
    adj = inputs.edges_to_adj(n, e)
    st = oracle.MemeticState(adj, k, p, K, seed=5, iters=60, use_scorer=use_scorer, d0=8, d=16, nl=3,
                             epochs=2, batch=5)
    prev_best = None
    for _ in range(3):
        fprime, pick = st.generation()
        assert np.all((pick >= 0) & (pick < K))
        # stored fitness and distances describe the stored population
        assert all(st.fP[i] == oracle.gamma(adj, k, st.P[i])[1] for i in range(p))
        assert np.array_equal(st.DP, oracle.distance_matrix(k, st.P, st.P))
        assert st.best_f[0] == oracle.gamma(adj, k, st.best_col)[1] <= fprime.min()
        if prev_best is not None:
            assert st.best_f[0] <= prev_best
        prev_best = st.best_f[0]
        # each offspring is a GPX child of i and one of its K nearest neighbours
        nbr = oracle.knn(st.DP, K)
        for i in range(p):
            j = nbr[i, pick[i]]
            child = oracle.gpx(k, st.P[i], st.P[j], seed=5, child_id=i * K + pick[i], gen=st.gen - 1)
            assert np.array_equal(child, st.SO[i])


@pytest.mark.parametrize("use_scorer", [0, 1])
def test_wvcp_memetic_generation_invariants(use_scorer):
    """Algorithm 1 for the WVCP: the stored fitness is the WVCP score of the stored (legal)
    colourings, the distances describe the population, the best-so-far is monotone and recounts,
    every f(S') is the score of a legal colouring or sum(w) + 1, and every offspring is the GPX
    child of i and one of its K nearest neighbours."""
    n, p, K = 30, 10, 3
    e = inputs.gnp(n, 0.3, seed=4)
    adj = inputs.edges_to_adj(n, e)
    w = inputs.weights(n, seed=4, hi=20)
    k = max(oracle.wvcp_greedy(adj, w, 6, i)[1] for i in range(p)) + 1
    fscale = 16
    phi0 = (fscale * k * int(w.max()) + n) // (2 * n)
    st = oracle.WvcpMemeticState(adj, w, k, p, K, seed=6, iters=40, max_ls=3, fscale=fscale, phi0=phi0,
                                 phi_last=fscale * 2 * int(w.max()), use_scorer=use_scorer, d0=8, d=16, nl=3,
                                 epochs=2, batch=4)
    assert all(oracle.wvcp_score(adj, w, k, c)[1] == 0 for c in st.P)
    prev = None
    for _ in range(3):
        fprime, pick = st.generation()
        assert np.all((fprime > 0) & (fprime <= w.sum() + 1))
        for i in range(p):  # a member without a legal result carries the fitness sum(w) + 1
            f, c = oracle.wvcp_score(adj, w, k, st.P[i])
            assert st.fP[i] == (f if c == 0 else w.sum() + 1)
        assert np.array_equal(st.DP, oracle.distance_matrix(k, st.P, st.P))
        bf, bc = oracle.wvcp_score(adj, w, k, st.best_col)
        assert bc == 0 and bf == st.best_f[0] <= fprime.min()
        if prev is not None:
            assert st.best_f[0] <= prev
        prev = st.best_f[0]
        nbr = oracle.knn(st.DP, K)
        for i in range(p):
            j = nbr[i, pick[i]]
            child = oracle.gpx(k, st.P[i], st.P[j], seed=6, child_id=i * K + pick[i], gen=st.gen - 1)
            assert np.array_equal(child, st.SO[i])
