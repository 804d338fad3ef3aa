"""GPU parity of whole memetic generations (Algorithm 1) against the oracle, through the C-ABI.
Random-GPX generations are integer work and must match bit for bit; learned generations match bit
for bit when the oracle selects offspring with the GPU's scores."""
import time

import numpy as np
import pytest

import oracle
from paper_2109_05948_gb300 import dlmcol, inputs

from gpu_util import device_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2109_05948_gb300 import build

    build.build()
    c = dlmcol.Context(0)
    yield c
    c.close()


def _get(ctx, mm, which, shape, dtype):
    t = torch.zeros(shape, dtype=dtype, device="cuda")
    dlmcol.dlm_memetic_get(ctx, mm, which, t)
    ctx.sync()
    return t.cpu().numpy()


def _compare(ctx, mm, st, p, n, K, step):
    assert np.array_equal(_get(ctx, mm, 0, (p, n), torch.int16), st.P), f"P at generation {step}"
    assert np.array_equal(_get(ctx, mm, 1, (p,), torch.int64), st.fP), f"f(P) at generation {step}"
    assert np.array_equal(_get(ctx, mm, 2, (p, p), torch.int16), st.DP), f"D(P) at generation {step}"
    assert np.array_equal(_get(ctx, mm, 3, (p, n), torch.int16), st.SO), f"S^O at generation {step}"
    assert np.array_equal(_get(ctx, mm, 4, (n,), torch.int16), st.best_col)


@pytest.mark.parametrize("n,k,p,K,iters,gens,seed", [(80, 5, 48, 6, 300, 3, 1), (130, 8, 40, 39, 200, 2, 2)])
def test_memetic_random_gpx_bitexact(ctx, n, k, p, K, iters, gens, seed):
    e, _ = inputs.planted(n, k, 0.4, seed=seed)
    adj = inputs.edges_to_adj(n, e)
    g = device_graph(ctx, n, e)
    prm = dlmcol.MemeticParams(k=k, p=p, K=K, iters=iters, tenure=dlmcol.COL_TENURE, use_scorer=0, epochs=0, batch=100,
                               lr=1e-3, seed=seed)
    mm = dlmcol.Memetic(ctx, g, prm)
    st = oracle.MemeticState(adj, k, p, K, seed=seed, iters=iters, use_scorer=0)
    _compare(ctx, mm, st, p, n, K, -1)
    with pytest.raises(dlmcol.DlmError):  # no generation has run yet
        dlmcol.dlm_memetic_found_ms(ctx, mm)
    for gen in range(gens):
        t0 = time.perf_counter()
        best = dlmcol.dlm_memetic_step(ctx, mm)
        wall_ms = (time.perf_counter() - t0) * 1e3
        # the best-so-far update ends inside the generation, after its local search
        assert 0.0 < dlmcol.dlm_memetic_found_ms(ctx, mm) <= wall_ms
        fprime, pick = st.generation()
        assert np.array_equal(_get(ctx, mm, 5, (p,), torch.int64), fprime)
        assert np.array_equal(_get(ctx, mm, 6, (p,), torch.int32), pick)
        assert best == st.best_f[0]
        _compare(ctx, mm, st, p, n, K, gen)
    mm.close()


def test_memetic_learned_selection_bitexact_with_gpu_scores(ctx):
    n, k, p, K, iters, seed = 60, 5, 32, 4, 200, 3
    e, _ = inputs.planted(n, k, 0.4, seed=seed)
    adj = inputs.edges_to_adj(n, e)
    g = device_graph(ctx, n, e)
    prm = dlmcol.MemeticParams(k=k, p=p, K=K, iters=iters, tenure=dlmcol.COL_TENURE, use_scorer=1, epochs=1, batch=16,
                               lr=1e-3, seed=seed)
    mm = dlmcol.Memetic(ctx, g, prm)
    st = oracle.MemeticState(adj, k, p, K, seed=seed, iters=iters, use_scorer=1, epochs=1, batch=16)
    for gen in range(2):
        dlmcol.dlm_memetic_step(ctx, mm)
        scores = _get(ctx, mm, 7, (p, K), torch.float32)
        assert np.all(np.isfinite(scores))
        fprime, pick = st.generation(ext_scores=scores)
        assert np.array_equal(_get(ctx, mm, 6, (p,), torch.int32), pick)
        assert np.array_equal(_get(ctx, mm, 5, (p,), torch.int64), fprime)
        _compare(ctx, mm, st, p, n, K, gen)
    mm.close()


def test_memetic_scorer_scores_match_oracle_after_training(ctx):
    """After one learned generation, the GPU's candidate scores equal the oracle network (FP64)
    evaluated with the GPU's trained parameters, within the scorer tolerance."""
    n, k, p, K, iters, seed = 60, 5, 32, 4, 150, 4
    e, _ = inputs.planted(n, k, 0.4, seed=seed)
    g = device_graph(ctx, n, e)
    prm = dlmcol.MemeticParams(k=k, p=p, K=K, iters=iters, tenure=dlmcol.COL_TENURE, use_scorer=1, epochs=2, batch=16,
                               lr=1e-3, seed=seed)
    mm = dlmcol.Memetic(ctx, g, prm)
    dlmcol.dlm_memetic_step(ctx, mm)
    scores = _get(ctx, mm, 7, (p, K), torch.float32)
    P = _get(ctx, mm, 0, (p, n), torch.int16)
    nparams = oracle.ScorerDims(n).nparams()
    th = _get(ctx, mm, 8, (nparams,), torch.float32).astype(np.float64)
    DP = _get(ctx, mm, 2, (p, p), torch.int16)
    nbr = oracle.knn(DP, K)
    kids = np.stack([oracle.gpx(k, P[i], P[nbr[i, j]], seed, i * K + j, 0) for i in range(p) for j in range(K)])
    ref = oracle.scorer_forward(oracle.ScorerDims(n), k, th, kids).reshape(p, K)
    rel = np.linalg.norm(scores - ref) / np.linalg.norm(ref)
    assert rel <= 1e-2
    mm.close()


def _state(ctx, mm, p, n, K, learned):
    out = [_get(ctx, mm, w, s, d) for w, s, d in [(0, (p, n), torch.int16), (1, (p,), torch.int64),
                                                   (2, (p, p), torch.int16), (3, (p, n), torch.int16),
                                                   (4, (n,), torch.int16), (5, (p,), torch.int64),
                                                   (6, (p,), torch.int32)]]
    if learned:
        out.append(_get(ctx, mm, 7, (p, K), torch.float32))
    return out


@pytest.mark.parametrize("learned", [0, 1])
def test_memetic_checkpoint_resume_and_determinism(ctx, learned):
    """Two objects with the same seed run identical generations; a third object loaded from the
    first one's checkpoint after two generations continues bit-identically (population, distances,
    offspring, best colouring, picks and, in the learned mode, candidate scores)."""
    n, k, p, K, iters, seed = 70, 5, 24, 4, 150, 8
    e, _ = inputs.planted(n, k, 0.4, seed=seed)
    g = device_graph(ctx, n, e)
    prm = dlmcol.MemeticParams(k=k, p=p, K=K, iters=iters, tenure=dlmcol.COL_TENURE, use_scorer=learned, epochs=1,
                               batch=8, lr=1e-3, seed=seed)
    a, b = dlmcol.Memetic(ctx, g, prm), dlmcol.Memetic(ctx, g, prm)
    for _ in range(2):
        fa, fb = dlmcol.dlm_memetic_step(ctx, a), dlmcol.dlm_memetic_step(ctx, b)
        assert fa == fb
        for x, y in zip(_state(ctx, a, p, n, K, learned), _state(ctx, b, p, n, K, learned)):
            assert np.array_equal(x, y)
    blob = dlmcol.dlm_memetic_save(ctx, a)
    c = dlmcol.Memetic(ctx, g, prm)
    dlmcol.dlm_memetic_load(ctx, c, blob)
    for _ in range(2):
        fa, fc = dlmcol.dlm_memetic_step(ctx, a), dlmcol.dlm_memetic_step(ctx, c)
        assert fa == fc
        for x, y in zip(_state(ctx, a, p, n, K, learned), _state(ctx, c, p, n, K, learned)):
            assert np.array_equal(x, y)
    # a checkpoint of another configuration is refused
    other = dlmcol.Memetic(ctx, g, dlmcol.MemeticParams(k=k, p=p + 2, K=K, iters=iters, tenure=dlmcol.COL_TENURE,
                                                        use_scorer=learned, epochs=1, batch=8, lr=1e-3, seed=seed))
    with pytest.raises(dlmcol.DlmError):
        dlmcol.dlm_memetic_load(ctx, other, blob)
    bad = blob.copy()
    bad[:8] = 0
    with pytest.raises(dlmcol.DlmError):
        dlmcol.dlm_memetic_load(ctx, c, bad)
    # same sizes, another seed, budget or graph: refused too (a resume must continue the same run)
    e2, _ = inputs.planted(n, k, 0.4, seed=seed + 1)
    g2 = device_graph(ctx, n, e2)
    others = [dlmcol.Memetic(ctx, g, dlmcol.MemeticParams(k=k, p=p, K=K, iters=iters, tenure=dlmcol.COL_TENURE,
                                                          use_scorer=learned, epochs=1, batch=8, lr=1e-3, seed=seed + 1)),
              dlmcol.Memetic(ctx, g, dlmcol.MemeticParams(k=k, p=p, K=K, iters=iters + 1, tenure=dlmcol.COL_TENURE,
                                                          use_scorer=learned, epochs=1, batch=8, lr=1e-3, seed=seed)),
              dlmcol.Memetic(ctx, g2, prm)]
    for o in others:
        with pytest.raises(dlmcol.DlmError):
            dlmcol.dlm_memetic_load(ctx, o, blob)
    for m in (a, b, c, other, *others):
        m.close()


def test_col_descend_matches_oracle_descent(ctx):
    """k-COL with decreasing k: the GPU descent stops at the same k, after the same numbers of
    generations, with the same legal colouring as a descent driven by the oracle generation by
    generation (random GPX, integer work throughout)."""
    n, k0, p, K, iters, seed, max_gens = 40, 6, 16, 4, 200, 5, 6
    e, _ = inputs.planted(n, 4, 0.5, seed=seed)
    adj = inputs.edges_to_adj(n, e)
    g = device_graph(ctx, n, e)
    prm = dlmcol.MemeticParams(k=k0, p=p, K=K, iters=iters, tenure=dlmcol.COL_TENURE, use_scorer=0, epochs=0,
                               batch=100, lr=1e-3, seed=seed)
    best = torch.zeros(n, dtype=torch.int16, device="cuda")
    kb, gens = dlmcol.dlm_col_descend(ctx, g, prm, max_gens, best)
    ref_k, ref_col = -1, None
    for k in range(k0, 1, -1):
        st = oracle.MemeticState(adj, k, p, K, seed=seed, iters=iters, use_scorer=0)
        solved, ran = False, 0
        for _ in range(max_gens):
            st.generation()
            ran += 1
            if st.best_f[0] == 0:
                solved = True
                break
        assert gens[k] == ran, k
        if not solved:
            break
        ref_k, ref_col = k, st.best_col.copy()
    assert kb == ref_k and kb >= 2
    b = best.cpu().numpy()
    assert np.array_equal(b, ref_col)
    assert int(np.sum(b[e[:, 0]] == b[e[:, 1]])) == 0 and int(b.max()) < kb


def test_learned_selection_gain_over_random_gpx(ctx):
    """What the trained network gains over the method without it (the ablation of section
    "Analysis of the contributions of deep learning", second parent drawn at random), on the
    learned workload's graph (planted 48-colourable, n = 1000, p = 0.5 across parts) at population
    2048, 2000 tabu iterations per generation, K = 32, 6 seeds per mode, up to 5 generations:
      * the network's predictions for the offspring it selects correlate with the conflicts those
        offspring reach after tabu search once it has trained on one generation (median Pearson
        over the seeds at generations 2 and 3 above 0.3; about 0 before any training);
      * the offspring it selects reach fewer conflicts than random GPX offspring of the same
        generation (median over seeds of the mean f(S') at generations 2 and 3);
      * the learned search needs no more generations to a legal colouring than random GPX.
    Wall time is not asserted: a learned generation also trains the network and scores 32
    candidates per individual (measured in bench.py --workload memetic)."""
    n, k, p, K, iters, seeds, gens = 1000, 48, 2048, 32, 2000, 6, 5
    e, _ = inputs.planted(n, k, 0.5, seed=0)
    g = device_graph(ctx, n, e)
    res = {0: [], 1: []}
    for learned in (1, 0):
        for sd in range(seeds):
            prm = dlmcol.MemeticParams(k=k, p=p, K=K, iters=iters, tenure=dlmcol.COL_TENURE, use_scorer=learned,
                                       epochs=5, batch=100, lr=1e-3, seed=500 + sd)
            mm = dlmcol.Memetic(ctx, g, prm)
            stats, reached = [], None
            for gi in range(gens):
                best = dlmcol.dlm_memetic_step(ctx, mm)
                stats.append(dlmcol.dlm_memetic_stats(ctx, mm))
                if best == 0 and reached is None:
                    reached = gi + 1
                    break
            res[learned].append((stats, reached if reached is not None else gens + 1))
            mm.close()

    def med_at(learned, key, gi):
        vals = [s[gi][key] for s, _ in res[learned] if len(s) > gi]
        return float(np.median(vals)) if vals else None

    for gi in (2, 3):
        pl = med_at(1, "pred_pearson", gi)
        fl, fr = med_at(1, "f_mean", gi), med_at(0, "f_mean", gi)
        if pl is not None:
            assert pl > 0.3, (gi, pl)
        if fl is not None and fr is not None:
            assert fl < fr, (gi, fl, fr)
    assert abs(med_at(1, "pred_pearson", 1)) < 0.3  # before the first training pays off
    assert np.median([r for _, r in res[1]]) <= np.median([r for _, r in res[0]])


def _wvcp_case(n, dens, seed, extra):
    e = inputs.gnp(n, dens, seed)
    w = inputs.weights(n, seed)
    adj = inputs.edges_to_adj(n, e)
    used = max(oracle.wvcp_greedy(adj, w, seed, i)[1] for i in range(64))
    return e, w, adj, used + extra


def _wvcp_phi(n, k, w):
    # the penalty schedule dlm_memetic_create documents: round(256 k max w / (2 |V|)), 256 * 2 max w
    return max(1, (256 * k * int(w.max()) + n) // (2 * n)), 256 * 2 * int(w.max())


@pytest.mark.parametrize("n,dens,p,K,iters,max_ls,gens,seed,extra",
                         [(60, 0.3, 24, 4, 120, 3, 2, 11, 3), (90, 0.5, 16, 15, 90, 4, 2, 12, 70)])
def test_wvcp_memetic_random_gpx_bitexact(ctx, n, dens, p, K, iters, max_ls, gens, seed, extra):
    """WVCP generations (greedy initial population, iterated feasible / infeasible tabu search,
    WVCP fitness) against the oracle, bit for bit; the second case has k above 64 colours."""
    e, w, adj, k = _wvcp_case(n, dens, seed, extra)
    g = device_graph(ctx, n, e, w)
    prm = dlmcol.MemeticParams(k=k, p=p, K=K, iters=iters, tenure=dlmcol.WVCP_TENURE, use_scorer=0, epochs=0,
                               batch=100, lr=1e-3, seed=seed, problem=1, max_ls=max_ls)
    mm = dlmcol.Memetic(ctx, g, prm)
    phi0, phi_last = _wvcp_phi(n, k, w)
    st = oracle.WvcpMemeticState(adj, w, k, p, K, seed, iters, max_ls, 256, phi0, phi_last, use_scorer=0)
    _compare(ctx, mm, st, p, n, K, -1)
    for gen in range(gens):
        best = dlmcol.dlm_memetic_step(ctx, mm)
        fprime, pick = st.generation()
        assert np.array_equal(_get(ctx, mm, 5, (p,), torch.int64), fprime)
        assert np.array_equal(_get(ctx, mm, 6, (p,), torch.int32), pick)
        assert best == st.best_f[0]
        _compare(ctx, mm, st, p, n, K, gen)
    mm.close()


@pytest.mark.parametrize("extra", [2, 100])
def test_wvcp_memetic_learned_bitexact_with_gpu_scores(ctx, extra):
    """Learned WVCP generations: with the GPU's candidate scores the oracle picks the same
    offspring and every array matches; extra = 100 puts k above 128 (three 64-row blocks of the
    scorer's colour rows)."""
    n, dens, p, K, iters, max_ls, seed = 70, 0.4, 16, 4, 80, 3, 13
    e, w, adj, k = _wvcp_case(n, dens, seed, extra)
    g = device_graph(ctx, n, e, w)
    prm = dlmcol.MemeticParams(k=k, p=p, K=K, iters=iters, tenure=dlmcol.WVCP_TENURE, use_scorer=1, epochs=1,
                               batch=8, lr=1e-3, seed=seed, problem=1, max_ls=max_ls)
    mm = dlmcol.Memetic(ctx, g, prm)
    phi0, phi_last = _wvcp_phi(n, k, w)
    st = oracle.WvcpMemeticState(adj, w, k, p, K, seed, iters, max_ls, 256, phi0, phi_last, use_scorer=1, epochs=1,
                                 batch=8)
    for gen in range(2):
        dlmcol.dlm_memetic_step(ctx, mm)
        scores = _get(ctx, mm, 7, (p, K), torch.float32)
        assert np.all(np.isfinite(scores))
        fprime, pick = st.generation(ext_scores=scores)
        assert np.array_equal(_get(ctx, mm, 6, (p,), torch.int32), pick)
        assert np.array_equal(_get(ctx, mm, 5, (p,), torch.int64), fprime)
        _compare(ctx, mm, st, p, n, K, gen)
    # the trained network's scores of the GPU's candidates against the oracle network (FP64) with the
    # GPU's parameters: selection-precision scores within the memetic's bf16 bound
    dlmcol.dlm_memetic_step(ctx, mm)
    nparams = oracle.ScorerDims(n).nparams()
    th = _get(ctx, mm, 8, (nparams,), torch.float32).astype(np.float64)
    scores = _get(ctx, mm, 7, (p, K), torch.float32)
    P = _get(ctx, mm, 0, (p, n), torch.int16)
    nbr = oracle.knn(_get(ctx, mm, 2, (p, p), torch.int16), K)
    kids = np.stack([oracle.gpx(k, P[i], P[nbr[i, j]], seed, i * K + j, 2) for i in range(p) for j in range(K)])
    ref = oracle.scorer_forward(oracle.ScorerDims(n), k, th, kids).reshape(p, K)
    rel = np.linalg.norm(scores - ref) / np.linalg.norm(ref)
    assert rel <= 1e-2
    mm.close()


def test_wvcp_memetic_rejects_bad_parameters(ctx):
    n = 40
    e = inputs.gnp(n, 0.3, 1)
    w = inputs.weights(n, 1)
    g_now = device_graph(ctx, n, e)
    g = device_graph(ctx, n, e, w)
    base = dict(p=8, K=2, iters=10, tenure=dlmcol.WVCP_TENURE, use_scorer=0, epochs=0, batch=8, lr=1e-3, seed=1,
                problem=1, max_ls=2)
    with pytest.raises(RuntimeError):
        dlmcol.Memetic(ctx, g_now, dlmcol.MemeticParams(k=20, **base))  # no weights
    with pytest.raises(RuntimeError):
        dlmcol.Memetic(ctx, g, dlmcol.MemeticParams(k=2, **base))  # the greedy needs more colours
    with pytest.raises(RuntimeError):
        dlmcol.Memetic(ctx, g, dlmcol.MemeticParams(k=256, **base))
    bad = dict(base, max_ls=0)
    with pytest.raises(RuntimeError):
        dlmcol.Memetic(ctx, g, dlmcol.MemeticParams(k=20, **bad))


def test_memetic_paper_size_network_selection(ctx):
    """use_scorer = 2 (the paper-size network with invariant batch normalisation, widths 10|V| ...
    |V|//2): generations bit-exact with the oracle selecting on the GPU's scores; the scores equal
    the FP64 network with the GPU's trained parameters and running statistics; a checkpoint resumes
    bit-identically."""
    from oracle import deepnet as dn

    n, k, p, K, iters, seed = 40, 5, 12, 3, 120, 5
    e, _ = inputs.planted(n, k, 0.4, seed=seed)
    adj = inputs.edges_to_adj(n, e)
    g = device_graph(ctx, n, e)
    prm = dlmcol.MemeticParams(k=k, p=p, K=K, iters=iters, tenure=dlmcol.COL_TENURE, use_scorer=2, epochs=2, batch=5,
                               lr=1e-3, seed=seed)
    mm = dlmcol.Memetic(ctx, g, prm)
    st = oracle.MemeticState(adj, k, p, K, seed=seed, iters=iters, use_scorer=1, epochs=1, batch=5)
    dims = dn.DeepDims(n, dn.paper_widths(n, "col"))
    for gen in range(2):
        dlmcol.dlm_memetic_step(ctx, mm)
        scores = _get(ctx, mm, 7, (p, K), torch.float32)
        assert np.all(np.isfinite(scores))
        fprime, pick = st.generation(ext_scores=scores)
        assert np.array_equal(_get(ctx, mm, 6, (p,), torch.int32), pick)
        assert np.array_equal(_get(ctx, mm, 5, (p,), torch.int64), fprime)
        _compare(ctx, mm, st, p, n, K, gen)
    th = _get(ctx, mm, 8, (dims.nparams(),), torch.float32).astype(np.float64)
    stats = _get(ctx, mm, 9, (dims.nstats(),), torch.float32).astype(np.float64)
    P = _get(ctx, mm, 0, (p, n), torch.int16)
    nbr = oracle.knn(_get(ctx, mm, 2, (p, p), torch.int16), K)
    kids = np.stack([oracle.gpx(k, P[i], P[nbr[i, j]], seed, i * K + j, 1) for i in range(p) for j in range(K)])
    ref = dn.forward(dims, k, th, kids, False, stats.copy()).reshape(p, K)
    bh = dims.view(th)["bh"][0]
    cg, cr = scores - bh, ref - bh
    floor = np.sqrt(np.mean(cr * cr))
    assert np.max(np.abs(cg - cr) / np.maximum(np.abs(cr), floor)) <= 1e-2
    # checkpoint and resume
    blob = dlmcol.dlm_memetic_save(ctx, mm)
    other = dlmcol.Memetic(ctx, g, prm)
    dlmcol.dlm_memetic_load(ctx, other, blob)
    fa, fb = dlmcol.dlm_memetic_step(ctx, mm), dlmcol.dlm_memetic_step(ctx, other)
    assert fa == fb
    for w, shp, dt in [(0, (p, n), torch.int16), (3, (p, n), torch.int16), (7, (p, K), torch.float32)]:
        assert np.array_equal(_get(ctx, mm, w, shp, dt), _get(ctx, other, w, shp, dt))
    mm.close()
    other.close()
