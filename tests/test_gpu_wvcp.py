"""GPU parity of the weighted vertex colouring path (randomised greedy initialisation and the
feasible/infeasible tabu search) against the oracle, through the C-ABI (integer work: bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_2109_05948_gb300 import dlmcol, inputs

from gpu_util import device_graph, oracle_pool

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


def _oracle_greedy(adj, w, seed, ind):
    n = adj.shape[0]
    col = np.zeros(n, np.int16)
    used = oracle.lib().oracle_wvcp_greedy(n, oracle._ptr(adj), oracle._ptr(w), seed, ind, oracle._ptr(col))
    return col, used


def _oracle_tabu(args):
    import oracle as o

    adj, w, k, col, iters, phi, seed, ind, gen, trace = args
    n = adj.shape[0]
    best = np.zeros(n, np.int16)
    bg, fc, mv = np.zeros(1, np.int64), np.zeros(2, np.int64), np.zeros(1, np.int64)
    tr = np.full((iters, 4), -7, np.int32) if trace else None
    rc = o.lib().oracle_wvcp_tabu(n, o._ptr(adj), o._ptr(w), k, o._ptr(col), iters, 9, 2, 10, phi, seed, ind, gen,
                                  o._ptr(best), o._ptr(bg), o._ptr(fc), o._ptr(mv), o._ptr(tr) if trace else None, 0)
    assert rc == 0
    return dict(best_col=best, best_g=int(bg[0]), f=int(fc[0]), c=int(fc[1]), moves=int(mv[0]), trace=tr)


def _case(n, p, seed):
    e = inputs.gnp(n, p, seed)
    adj = inputs.edges_to_adj(n, e)
    w = inputs.weights(n, seed)
    return e, adj, w


@pytest.mark.parametrize("n,p,seed,pop", [(60, 0.5, 1, 8), (200, 0.3, 2, 5), (500, 0.5, 3, 3)])
def test_greedy_matches_oracle(ctx, n, p, seed, pop):
    e, adj, w = _case(n, p, seed)
    g = device_graph(ctx, n, e, w)
    col = torch.zeros((pop, n), dtype=torch.int16, device="cuda")
    used = torch.zeros(pop, dtype=torch.int32, device="cuda")
    dlmcol.dlm_wvcp_greedy(ctx, g, pop, seed, 4, col, used)
    ctx.sync()
    for i in range(pop):
        ref, u = _oracle_greedy(adj, w, seed, 4 + i)
        assert np.array_equal(col[i].cpu().numpy(), ref) and used[i].item() == u


def _run_gpu(ctx, g, k, starts, iters, phi, seed, gen, trace=False, entry_bits=0):
    pop, n = starts.shape
    col = torch.from_numpy(starts.copy()).cuda()
    bg = torch.zeros(pop, dtype=torch.int64, device="cuda")
    fc = torch.zeros((pop, 2), dtype=torch.int64, device="cuda")
    mv = torch.zeros(pop, dtype=torch.int64, device="cuda")
    tr = torch.full((pop, iters, 4), -7, dtype=torch.int32, device="cuda") if trace else None
    dlmcol.dlm_wvcp_tabu_batch_ex(ctx, g, k, pop, col, bg, fc, mv, iters, dlmcol.WVCP_TENURE, phi, seed, gen, 0, tr,
                                  entry_bits)
    ctx.sync()
    return col.cpu().numpy(), bg.cpu().numpy(), fc.cpu().numpy(), mv.cpu().numpy(), (tr.cpu().numpy() if trace else None)


@pytest.mark.parametrize("entry_bits", [8, 16])
@pytest.mark.parametrize("n,p,seed,iters,legal_start", [(40, 0.5, 1, 400, True), (90, 0.3, 2, 600, False),
                                                         (150, 0.6, 3, 500, True), (63, 0.9, 4, 300, False)])
def test_wvcp_tabu_bitexact(ctx, n, p, seed, iters, legal_start, entry_bits):
    e, adj, w = _case(n, p, seed)
    g = device_graph(ctx, n, e, w)
    greedy = [_oracle_greedy(adj, w, seed, i) for i in range(4)]
    k = max(u for _, u in greedy)
    starts = np.stack([c for c, _ in greedy]) if legal_start else inputs.random_colorings(4, n, k, seed=seed)
    phi = 2 * int(w.max())
    col, bg, fc, mv, tr = _run_gpu(ctx, g, k, starts, iters, phi, seed, 3, trace=True, entry_bits=entry_bits)
    for i in range(4):
        r = _oracle_tabu((adj, w, k, starts[i], iters, phi, seed, i, 3, True))
        assert np.array_equal(tr[i], r["trace"]), f"first divergence at {int(np.argmax(np.any(tr[i] != r['trace'], 1)))}"
        assert (bg[i], fc[i, 0], fc[i, 1], mv[i]) == (r["best_g"], r["f"], r["c"], r["moves"])
        assert np.array_equal(col[i], r["best_col"])


def test_wvcp_unit_weights_and_small_phi(ctx):
    n = 80
    e = inputs.gnp(n, 0.4, 7)
    adj = inputs.edges_to_adj(n, e)
    w = np.ones(n, np.int32)
    g = device_graph(ctx, n, e, w)
    k = 12
    starts = inputs.random_colorings(3, n, k, seed=5)
    col, bg, fc, mv, _ = _run_gpu(ctx, g, k, starts, 500, 1, 9, 0)
    for i in range(3):
        r = _oracle_tabu((adj, w, k, starts[i], 500, 1, 9, i, 0, False))
        assert (bg[i], fc[i, 0], fc[i, 1], mv[i]) == (r["best_g"], r["f"], r["c"], r["moves"])
        assert np.array_equal(col[i], r["best_col"])


def test_wvcp_rejects_bad_input(ctx):
    n = 30
    e = inputs.gnp(n, 0.3, 1)
    g_now = device_graph(ctx, n, e)  # no weights
    col = torch.zeros((1, n), dtype=torch.int16, device="cuda")
    bg = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(dlmcol.DlmError):
        dlmcol.dlm_wvcp_tabu_batch(ctx, g_now, 4, 1, col, bg, None, None, 10, dlmcol.WVCP_TENURE, 2)
    g = device_graph(ctx, n, e, inputs.weights(n, 1))
    with pytest.raises(dlmcol.DlmError):
        dlmcol.dlm_wvcp_tabu_batch(ctx, g, 300, 1, col, bg, None, None, 10, dlmcol.WVCP_TENURE, 2)
    col[0, 3] = 9
    dlmcol.dlm_wvcp_tabu_batch(ctx, g, 5, 1, col, bg, None, None, 10, dlmcol.WVCP_TENURE, 2)
    with pytest.raises(dlmcol.DlmError):
        ctx.sync()


def test_wvcp_full_size_sampled(ctx):
    """The weighted workload: G(1000, 0.5), weights 1..100, k from the greedy initialisation,
    phi = 2 max w. The automatic entry size is u8 (the whole conflict table in shared memory);
    forced u16 entries spill colours into the CTA's global slab and give the same results. Two
    individuals are replayed by the oracle over 1500 iterations."""
    n, pop, iters = 1000, 160, 1500
    e, adj, w = _case(n, 0.5, 0)
    g = device_graph(ctx, n, e, w)
    col = torch.zeros((pop, n), dtype=torch.int16, device="cuda")
    used = torch.zeros(pop, dtype=torch.int32, device="cuda")
    dlmcol.dlm_wvcp_greedy(ctx, g, pop, 0, 0, col, used)
    ctx.sync()
    k = int(used.max().item())
    starts = col.cpu().numpy()
    phi = 2 * int(w.max())
    assert dlmcol.dlm_wvcp_entry_bits(ctx, g, k) == 8
    gcol, bg, fc, mv, _ = _run_gpu(ctx, g, k, starts, iters, phi, 0, 0)
    wide = _run_gpu(ctx, g, k, starts, iters, phi, 0, 0, entry_bits=16)
    for a, b in zip((gcol, bg, fc, mv), wide[:4]):
        assert np.array_equal(a, b)
    # every individual: the reported f and c recount from the returned colouring
    for i in range(0, pop, 17):
        c_i = gcol[i]
        conf = int(np.sum(c_i[e[:, 0]] == c_i[e[:, 1]]))
        f = sum(int(w[c_i == q].max()) for q in range(k) if np.any(c_i == q))
        assert (fc[i, 0], fc[i, 1], bg[i]) == (f, conf, f + phi * conf)
    refs = oracle_pool().map(_oracle_tabu, [(adj, w, k, starts[i], iters, phi, 0, i, 0, False) for i in (0, pop - 1)])
    for i, r in zip((0, pop - 1), refs):
        assert (bg[i], fc[i, 0], fc[i, 1], mv[i]) == (r["best_g"], r["f"], r["c"], r["moves"])
        assert np.array_equal(gcol[i], r["best_col"])


def _oracle_iterated(args):
    import oracle as o

    adj, w, k, col, iters, max_ls, fscale, phi0, phi_last, seed, ind, gen = args
    return o.wvcp_iterated(adj, w, k, col, iters, max_ls, fscale, phi0, phi_last, seed, ind, gen)


@pytest.mark.parametrize("n,p,seed,iters,max_ls,legal_start", [(50, 0.5, 1, 200, 10, True), (90, 0.4, 2, 150, 4, False),
                                                                (40, 0.6, 3, 100, 1, False), (120, 0.5, 4, 120, 2, True)])
def test_wvcp_iterated_matches_oracle(ctx, n, p, seed, iters, max_ls, legal_start):
    """Algorithm 2 on the GPU: the best legal colouring and its f (or -1) and the last search's best
    colouring equal the oracle's for every individual (fixed-point phi, resolution 1/256)."""
    e, adj, w = _case(n, p, seed)
    g = device_graph(ctx, n, e, w)
    pop = 5
    greedy = [_oracle_greedy(adj, w, seed, i) for i in range(pop)]
    k = max(u for _, u in greedy)
    starts = np.stack([c for c, _ in greedy]) if legal_start else inputs.random_colorings(pop, n, k, seed=seed)
    fscale = 256
    phi0 = (fscale * k * int(w.max()) + n) // (2 * n)
    phi_last = fscale * 2 * int(w.max())
    col = torch.from_numpy(starts.copy()).cuda()
    best_col = torch.zeros_like(col)
    best_f = torch.zeros(pop, dtype=torch.int64, device="cuda")
    dlmcol.dlm_wvcp_iterated(ctx, g, k, pop, col, best_col, best_f, iters, max_ls, dlmcol.WVCP_TENURE, fscale, phi0,
                             phi_last, seed, 2, 0)
    ctx.sync()
    refs = oracle_pool().map(_oracle_iterated, [(adj, w, k, starts[i], iters, max_ls, fscale, phi0, phi_last, seed, i, 2)
                                                for i in range(pop)])
    bf, bc = best_f.cpu().numpy(), best_col.cpu().numpy()
    for i, r in enumerate(refs):
        assert bf[i] == r["best_f"], i
        assert np.array_equal(bc[i], r["best_col"]), i


def test_wvcp_iterated_rejects_overflowing_schedule(ctx):
    n = 30
    e = inputs.gnp(n, 0.5, 1)
    g = device_graph(ctx, n, e, inputs.weights(n, 1))
    col = torch.zeros((1, n), dtype=torch.int16, device="cuda")
    bf = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(dlmcol.DlmError):  # phi0 doubled eight times overflows the 32-bit keys
        dlmcol.dlm_wvcp_iterated(ctx, g, 5, 1, col, col.clone(), bf, 10, 10, dlmcol.WVCP_TENURE, 256, 1 << 20, 1)


def _oracle_vs_gpu(ctx, e, adj, w, k, starts, iters, phi, entry_bits):
    n = adj.shape[0]
    g = device_graph(ctx, n, e, w)
    col, bg, fc, mv, tr = _run_gpu(ctx, g, k, starts, iters, phi, 5, 1, trace=True, entry_bits=entry_bits)
    for i in range(starts.shape[0]):
        r = _oracle_tabu((adj, w, k, starts[i], iters, phi, 5, i, 1, True))
        assert np.array_equal(tr[i], r["trace"]), f"first divergence at {int(np.argmax(np.any(tr[i] != r['trace'], 1)))}"
        assert (bg[i], fc[i, 0], fc[i, 1], mv[i]) == (r["best_g"], r["f"], r["c"], r["moves"])
        assert np.array_equal(col[i], r["best_col"])
    return tr


@pytest.mark.parametrize("entry_bits", [0, 8])
def test_wvcp_u8_gives_up_a_start_class_above_255(ctx, entry_bits):
    """A star: the hub (weight 200, colour 1) has 257 leaves (weight 50) in colour 0, so
    gamma[hub][0] = 257 does not fit a u8 entry. Read as 1, it would make the hub's move to colour 0
    the best (delta -49 at phi = 1); the true best moves the hub to colour 2 (delta -19). The u8
    search gives the individual up at set-up and the u16 pass reproduces the oracle's trace; a
    second individual with small classes stays with the u8 search."""
    n = 277
    e = np.array([(0, v) for v in range(1, 258)] + [(258 + i, 259 + i) for i in range(18)], np.int32)
    adj = inputs.edges_to_adj(n, e)
    w = np.full(n, 50, np.int32)
    w[0] = 200
    w[258:] = np.arange(1, 20)
    k = 4
    star = np.zeros(n, np.int16)
    star[0] = 1
    star[258:] = 2 + (np.arange(19) % 2)
    small = inputs.random_colorings(1, n, k, seed=3)[0]
    tr = _oracle_vs_gpu(ctx, e, adj, w, k, np.stack([star, small]), 300, 1, entry_bits)
    assert tuple(tr[0, 0, :3]) == (0, 2, -19)


def test_wvcp_u8_gives_up_when_a_class_grows_past_255(ctx):
    """Colour 0 starts with 253 vertices of weight 100; 20 singleton classes of weights 60, 59, ...
    each merge into it in turn (the unique best move: the class maximum stays 100). The third merge
    would make 256 vertices: the u8 search gives up there and the u16 pass, from the start
    colouring, reproduces the oracle's whole trace."""
    m = 20
    n = 253 + m
    rng = np.random.default_rng(4)
    e = np.array([(253 + i, 253 + j) for i in range(m) for j in range(i + 1, m) if rng.random() < 0.3], np.int32)
    adj = inputs.edges_to_adj(n, e)
    w = np.full(n, 100, np.int32)
    w[253:] = 60 - np.arange(m)
    k = m + 3
    start = np.zeros(n, np.int16)
    start[253:] = 1 + np.arange(m)
    tr = _oracle_vs_gpu(ctx, e, adj, w, k, start[None, :], 400, 2 * 100, 8)
    assert [tuple(tr[0, i, :2]) for i in range(3)] == [(253, 0), (254, 0), (255, 0)]


def test_wvcp_entry_bits_choice(ctx):
    e, adj, w = _case(1000, 0.5, 0)
    g = device_graph(ctx, 1000, e, w)
    assert dlmcol.dlm_wvcp_entry_bits(ctx, g, 145) == 8
    assert dlmcol.dlm_wvcp_entry_bits(ctx, g, 40) == 16  # u16 keeps the whole table on chip
    col = torch.zeros((1, 1000), dtype=torch.int16, device="cuda")
    bg = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(dlmcol.DlmError):  # 255 colours of u8 entries do not fit
        dlmcol.dlm_wvcp_tabu_batch_ex(ctx, g, 255, 1, col, bg, None, None, 10, dlmcol.WVCP_TENURE, 2, entry_bits=8)
    with pytest.raises(dlmcol.DlmError):
        dlmcol.dlm_wvcp_tabu_batch_ex(ctx, g, 40, 1, col, bg, None, None, 10, dlmcol.WVCP_TENURE, 2, entry_bits=12)
