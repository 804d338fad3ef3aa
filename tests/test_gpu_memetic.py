"""GPU parity of whole memetic generations (Algorithm 1) against the oracle, through the C-ABI.
Random-GPX generations are integer work and must match bit for bit; learned generations match bit
for bit when the oracle selects offspring with the GPU's scores."""
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
    for gen in range(gens):
        best = dlmcol.dlm_memetic_step(ctx, mm)
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
    for m in (a, b, c, other):
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
