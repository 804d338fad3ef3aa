"""GPU parity of GPX, distances, pool update and K-nearest-neighbour matching against the oracle,
through the C-ABI (all integer work: bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_2109_05948_gb300 import dlmcol, inputs

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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,k,pop,m", [(300, 20, 50, 200), (1000, 48, 64, 300), (97, 101, 9, 40), (2048, 7, 4, 8),
                                       (1, 3, 2, 3)])
def test_gpx_matches_oracle(ctx, n, k, pop, m):
    rng = np.random.default_rng(n + k)
    parents = inputs.random_colorings(pop, n, k, seed=n)
    pairs = rng.integers(0, pop, size=(m, 2)).astype(np.int32)
    pairs[: min(m, 3), 1] = pairs[: min(m, 3), 0]  # identical parents
    cid = rng.integers(0, 2**32, size=m, dtype=np.uint64).astype(np.uint32)
    out = torch.zeros((m, n), dtype=torch.int16, device="cuda")
    dlmcol.dlm_gpx_batch(ctx, n, k, _cuda(parents), pop, _cuda(pairs), _cuda(cid), m, out, 77, 5)
    ctx.sync()
    got = out.cpu().numpy()
    for t in range(m):
        ref = oracle.gpx(k, parents[pairs[t, 0]], parents[pairs[t, 1]], seed=77, child_id=int(cid[t]), gen=5)
        assert np.array_equal(got[t], ref), t


def test_gpx_default_child_ids_and_bad_pairs(ctx):
    n, k, pop = 120, 9, 6
    parents = inputs.random_colorings(pop, n, k, seed=1)
    pairs = np.array([[0, 1], [2, 3], [5, 4]], np.int32)
    out = torch.zeros((3, n), dtype=torch.int16, device="cuda")
    dlmcol.dlm_gpx_batch(ctx, n, k, _cuda(parents), pop, _cuda(pairs), None, 3, out, 1, 0)
    ctx.sync()
    for t in range(3):
        assert np.array_equal(out[t].cpu().numpy(), oracle.gpx(k, parents[pairs[t, 0]], parents[pairs[t, 1]], 1, t, 0))
    bad = np.array([[0, 6]], np.int32)
    dlmcol.dlm_gpx_batch(ctx, n, k, _cuda(parents), pop, _cuda(bad), None, 1, out, 1, 0)
    with pytest.raises(dlmcol.DlmError):
        ctx.sync()


@pytest.mark.parametrize("method", [None, 1, 2, 3])
@pytest.mark.parametrize("n,k,a,b", [(257, 33, 40, 70), (1000, 48, 17, 130), (64, 128, 5, 9), (3, 2, 4, 4),
                                     (1000, 144, 9, 150), (2048, 255, 4, 70), (1001, 97, 6, 66)])
def test_distance_matches_oracle(ctx, n, k, a, b, method):
    if method == 3 and k > 128:  # the tensor-core path holds a pair's classes in one 128-row tile
        D = torch.zeros((a, b), dtype=torch.int16, device="cuda")
        X = _cuda(inputs.random_colorings(a, n, k, seed=a))
        with pytest.raises(dlmcol.DlmError):
            dlmcol.dlm_distance_batch(ctx, n, k, X, a, X, a, D, b, 0, method=3)
        return
    X = inputs.random_colorings(a, n, k, seed=a)
    Y = inputs.random_colorings(b, n, k, seed=b + 1)
    Y[0] = X[0]  # a zero distance
    Y[1] = np.random.default_rng(b).permutation(k)[X[min(1, a - 1)]]  # a relabelling: zero distance
    Y[2] = 0  # one class holding every vertex: a count of n
    if b > 3:
        Y[3] = X[0] % 2  # two classes
    ld = b + 3
    D = torch.full((a, ld), -1, dtype=torch.int16, device="cuda")
    dlmcol.dlm_distance_batch(ctx, n, k, _cuda(X), a, _cuda(Y), b, D, ld, 0, method=method)
    ctx.sync()
    got = D.cpu().numpy()
    assert np.array_equal(got[:, :b], oracle.distance_matrix(k, X, Y))
    assert np.all(got[:, b:] == -1)


@pytest.mark.parametrize("method", [None, 1])
def test_distance_large_classes(ctx, method):
    """Rows of X with a class above 255 vertices (their overlap counts need more than a byte) beside
    rows without, in one launch and in the upper-triangle form."""
    n, k, a, b = 1000, 48, 12, 140
    X = inputs.random_colorings(a, n, k, seed=5)
    X[1] = 0  # one class of n vertices
    X[4] = X[4] % 3  # three classes of about 333
    X[7, :600] = 5  # one class of at least 600
    X[10, :256] = 9  # one class of at least 256
    Y = inputs.random_colorings(b, n, k, seed=6)
    Y[0], Y[1], Y[2], Y[3] = X[1], X[4], 0, X[7]
    D = torch.full((a, b), -1, dtype=torch.int16, device="cuda")
    dlmcol.dlm_distance_batch(ctx, n, k, _cuda(X), a, _cuda(Y), b, D, b, 0, method=method)
    ctx.sync()
    assert np.array_equal(D.cpu().numpy(), oracle.distance_matrix(k, X, Y))
    Z = inputs.random_colorings(70, 600, 2, seed=7)  # two classes of about 300 in every row
    Z[5:9] = np.arange(600) % 2  # rows at distance 0 from each other
    D2 = torch.full((70, 70), -1, dtype=torch.int16, device="cuda")
    dlmcol.dlm_distance_batch(ctx, 600, 2, _cuda(Z), 70, _cuda(Z), 70, D2, 70, 1, method=method)
    ctx.sync()
    got, ref = D2.cpu().numpy(), oracle.distance_matrix(2, Z, Z)
    iu = np.triu_indices(70, 1)
    assert np.array_equal(got[iu], ref[iu])
    assert np.all(got[np.tril_indices(70)] == -1)


@pytest.mark.parametrize("method", [1, 2, 3])
@pytest.mark.parametrize("n,k,a", [(200, 12, 50), (300, 120, 70)])
def test_distance_upper_triangle(ctx, n, k, a, method):
    X = inputs.random_colorings(a, n, k, seed=3)
    D = torch.full((a, a), -1, dtype=torch.int16, device="cuda")
    dlmcol.dlm_distance_batch(ctx, n, k, _cuda(X), a, _cuda(X), a, D, a, 1, method=method)
    ctx.sync()
    got = D.cpu().numpy()
    ref = oracle.distance_matrix(k, X, X)
    iu = np.triu_indices(a, 1)
    assert np.array_equal(got[iu], ref[iu])
    assert np.all(got[np.tril_indices(a)] == -1)


@pytest.mark.parametrize("n,k,a,b", [(60, 5, 7, 9), (257, 33, 6, 11), (1000, 48, 3, 20), (300, 128, 2, 5),
                                     (130, 70, 4, 4), (5, 2, 3, 3)])
def test_distance_exact_matches_oracle(ctx, n, k, a, b):
    """The exact (Hungarian) distance equals the oracle's assignment-solver value on random pairs,
    relabellings (0), partners recoloured in a few vertices and partners far from one matching."""
    X = inputs.random_colorings(a, n, k, seed=a + 100)
    Y = inputs.random_colorings(b, n, k, seed=b + 200)
    Y[0] = np.random.default_rng(1).permutation(k)[X[0]]
    Y[1] = X[min(1, a - 1)].copy()
    Y[1][: min(n, 7)] = (Y[1][: min(n, 7)] + 1) % k
    Y[2] = 0
    ld = b + 1
    D = torch.full((a, ld), -1, dtype=torch.int16, device="cuda")
    dlmcol.dlm_distance_exact_batch(ctx, n, k, _cuda(X), a, _cuda(Y), b, D, ld, 0)
    ctx.sync()
    got = D.cpu().numpy()
    ref = oracle.distance_exact_matrix(k, X, Y)
    assert np.array_equal(got[:, :b], ref)
    assert np.all(got[:, b:] == -1)
    # the approximation is a lower bound of the exact value
    assert np.all(oracle.distance_matrix(k, X, Y) <= ref)


def test_distance_exact_upper_and_limits(ctx):
    n, k, a = 200, 20, 12
    X = inputs.random_colorings(a, n, k, seed=5)
    D = torch.full((a, a), -1, dtype=torch.int16, device="cuda")
    dlmcol.dlm_distance_exact_batch(ctx, n, k, _cuda(X), a, _cuda(X), a, D, a, 1)
    ctx.sync()
    got = D.cpu().numpy()
    ref = oracle.distance_exact_matrix(k, X, X)
    iu = np.triu_indices(a, 1)
    assert np.array_equal(got[iu], ref[iu])
    assert np.all(got[np.tril_indices(a)] == -1)
    with pytest.raises(dlmcol.DlmError):
        dlmcol.dlm_distance_exact_batch(ctx, n, 129, _cuda(X), a, _cuda(X), a, D, a, 0)


def _random_pool_case(p, n, seed, spread):
    rng = np.random.default_rng(seed)
    m = 2 * p
    D = rng.integers(0, spread, size=(m, m))
    D = np.triu(D, 1)
    D = (D + D.T).astype(np.int16)
    fit = rng.integers(0, 30, size=m).astype(np.int64)
    return fit, D


@pytest.mark.parametrize("p,n,seed,spread", [(64, 100, 0, 25), (300, 500, 1, 120), (33, 50, 2, 6), (1, 10, 3, 5),
                                             (8192, 1000, 4, 300),
                                             (700, 100, 5, 120),       # two blocks of 1024, the last ragged
                                             (2048, 1000, 6, 2000),    # few close pairs, four blocks
                                             (4100, 10, 7, 32000)])    # p kept in the middle of block 4
def test_pool_update_matches_oracle(ctx, p, n, seed, spread):
    """The kept candidates and their order equal the oracle's one-at-a-time greedy visit, with and
    without a fill, within one block of 1024 candidates and across several."""
    fit, D = _random_pool_case(p, n, seed, spread)
    sel = torch.zeros(p, dtype=torch.int32, device="cuda")
    dlmcol.dlm_pool_update(ctx, p, n, _cuda(fit), _cuda(D), sel)
    ctx.sync()
    assert np.array_equal(sel.cpu().numpy(), oracle.pool_update(p, n, fit, D))


@pytest.mark.parametrize("p,K,seed", [(300, 16, 0), (40, 39, 1), (8192, 32, 2), (2, 1, 3)])
def test_knn_matches_oracle(ctx, p, K, seed):
    rng = np.random.default_rng(seed)
    D = rng.integers(0, 60, size=(p, p))
    D = (np.triu(D, 1) + np.triu(D, 1).T).astype(np.int16)
    nbr = torch.zeros((p, K), dtype=torch.int32, device="cuda")
    dlmcol.dlm_knn(ctx, p, _cuda(D), K, nbr)
    ctx.sync()
    got = nbr.cpu().numpy()
    if p <= 300:
        assert np.array_equal(got, oracle.knn(D, K))
    else:  # the full-size matrix: sampled rows against a library sort
        for i in [0, 1, p // 2, p - 1]:
            js = np.array([j for j in range(p) if j != i])
            ref = js[np.argsort(D[i, js], kind="stable")][:K]
            assert np.array_equal(got[i], ref)


def test_knn_rejects_bad_k(ctx):
    D = torch.zeros((4, 4), dtype=torch.int16, device="cuda")
    nbr = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(dlmcol.DlmError):
        dlmcol.dlm_knn(ctx, 4, D, 4, nbr)


def test_distance_and_gpx_full_size_sampled(ctx):
    """The learned workload's sizes, in the launches the population bench times: P x P' and the
    upper triangle of P' x P' over 8192 colourings each (n = 1000, k = 48), and GPX for
    8192 x 32 parent pairs. Sampled rows of D and sampled children equal the oracle's."""
    n, k, p, K = 1000, 48, 8192, 32
    P = inputs.random_colorings(p, n, k, seed=21)
    Sp = inputs.random_colorings(p, n, k, seed=22)
    Sp[5] = P[7]  # a zero distance inside the sampled rows
    m = 2 * p
    dP, dSp = _cuda(P), _cuda(Sp)
    D = torch.full((m, m), -1, dtype=torch.int16, device="cuda")
    dlmcol.dlm_distance_batch(ctx, n, k, dP, p, dSp, p, D[:, p:], m, 0)
    dlmcol.dlm_distance_batch(ctx, n, k, dSp, p, dSp, p, D[p:, p:], m, 1)
    ctx.sync()
    rows = [0, 7, 4095, p - 1]
    for i in rows:
        got = D[i, p:].cpu().numpy()
        assert np.array_equal(got, oracle.distance_matrix(k, P[i:i + 1], Sp)[0]), i
        assert got[5] == 0 or i != 7
        up = D[p + i, p:].cpu().numpy()
        ref = oracle.distance_matrix(k, Sp[i:i + 1], Sp)[0]
        assert np.array_equal(up[i + 1:], ref[i + 1:]), i
        assert np.all(up[: i + 1] == -1), i
    # GPX: child t = i K + j of parents (i, nbr[i][j]) with random neighbours
    rng = np.random.default_rng(23)
    nbr = rng.integers(0, p, size=(p, K)).astype(np.int32)
    pairs = np.stack([np.repeat(np.arange(p, dtype=np.int32), K), nbr.reshape(-1)], 1)
    kids = torch.zeros((p * K, n), dtype=torch.int16, device="cuda")
    dlmcol.dlm_gpx_batch(ctx, n, k, dP, p, _cuda(pairs), None, p * K, kids, 31, 2)
    ctx.sync()
    for t in [0, 1, 31, 32, 131071, 200003, p * K - 1]:
        ref = oracle.gpx(k, P[pairs[t, 0]], P[pairs[t, 1]], seed=31, child_id=t, gen=2)
        assert np.array_equal(kids[t].cpu().numpy(), ref), t
